// k_build.cu -- tree construction on the GPU (§2.1, App. A, App. B).
//
//  frame + keys   per-system bounding box (order-preserving 64-bit atomics),
//                 frame (origin, power-of-two side L), 60-bit Morton keys;
//                 with a key depth D > 20 (App. B: longer keys lift the
//                 20-level limit) a second word holds levels 21..D.
//  sort           stable LSD radix sort of (key, index), 8-bit digits, one
//                 upsweep histogram for all passes and one pass kernel per
//                 digit with decoupled look-back (bounded waits).  A forest
//                 adds digits of the system id as the most significant ones.
//                 Deeper keys sort their low word first, then gather the
//                 60-bit word into the current order and sort by it.
//  move           gather of the bodies into key order, split into two floats.
//  cells          the paper's level loop (mask keys of unfinished bodies,
//                 group equal masked keys, cells of <= N_leaf bodies become
//                 leaves) computed for all 21 levels at once: a body's cell at
//                 level k holds more than N bodies iff some run of N+1
//                 consecutive sorted keys around it shares k levels, so each
//                 body learns its leaf level from a sliding window over its
//                 neighbours; the levels at which it starts a cell follow from
//                 its common prefix with the previous key.  One prefix sum over
//                 per-warp, per-level counts places every cell in (level, key)
//                 order and every group in body order; links come from binary
//                 searches in the sorted keys and the level-ordered cells.
#include <cuda_runtime.h>

#include "bh_internal.cuh"

namespace bh {

namespace {

constexpr int kBlock = 256;

// Order-preserving image of a double's bits as an unsigned integer (any
// non-NaN: x < y iff ord(x) < ord(y); -0 sorts just below +0).
__device__ __forceinline__ unsigned long long ord_bits(unsigned long long b) {
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ bool finite_bits(unsigned long long b) {
  return ((b >> 52) & 0x7ffull) != 0x7ffull;
}
__device__ __forceinline__ double double_of(unsigned long long o) {
  unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
  return __longlong_as_double((long long)b);
}

// --------------------------------------------------------------- reset
__global__ void k_reset(unsigned long long *minmax, int S, uint32_t *ticket) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 6 * S) minmax[t] = (t % 6 < 3) ? ~0ull : 0ull;
  if (t == 0) *ticket = 0;
}

// ---------------------------------------------------- bounding box + frame
// Each block reduces 4*256 consecutive bodies; a warp whose bodies share one
// system reduces in registers, otherwise its lanes update the system directly.
// The last block to finish turns min/max into the frame of every system.
template <bool FOREST>
__global__ void __launch_bounds__(kBlock) k_bbox(const double *__restrict__ pos, const double *__restrict__ mass,
                                                 int n, const int32_t *__restrict__ offs, int S,
                                                 unsigned long long *minmax, uint32_t *ticket, Frame *frame,
                                                 FrameF *framef, int32_t *status) {
  __shared__ unsigned long long s_v[kBlock / 32][6];
  __shared__ int s_sys[kBlock / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int base = blockIdx.x * (4 * kBlock);
  // min/max on the order-preserving integer images of the coordinates: exact,
  // and integer work (the GPU's FP64 rate is a small fraction of its FP32 rate)
  unsigned long long v[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
  int my_sys = -1;
  bool bad = false;
  for (int j = 0; j < 4; ++j) {
    int i = base + threadIdx.x + j * kBlock;
    if (i >= n) break;
    const unsigned long long x0 = (unsigned long long)__double_as_longlong(pos[3 * (size_t)i]);
    const unsigned long long x1 = (unsigned long long)__double_as_longlong(pos[3 * (size_t)i + 1]);
    const unsigned long long x2 = (unsigned long long)__double_as_longlong(pos[3 * (size_t)i + 2]);
    const unsigned long long m = (unsigned long long)__double_as_longlong(mass[i]);
    bad |= !(finite_bits(x0) && finite_bits(x1) && finite_bits(x2) && finite_bits(m));
    int s = FOREST ? sys_of(offs, S, i) : 0;
    if (my_sys >= 0 && s != my_sys) {
      // body of another system: flush what we have and start again
      for (int a = 0; a < 3; ++a) {
        atomicMin(&minmax[6 * my_sys + a], v[a]);
        atomicMax(&minmax[6 * my_sys + 3 + a], v[3 + a]);
      }
      v[0] = v[1] = v[2] = ~0ull;
      v[3] = v[4] = v[5] = 0ull;
    }
    my_sys = s;
    const unsigned long long o0 = ord_bits(x0), o1 = ord_bits(x1), o2 = ord_bits(x2);
    v[0] = min(v[0], o0); v[1] = min(v[1], o1); v[2] = min(v[2], o2);
    v[3] = max(v[3], o0); v[4] = max(v[4], o1); v[5] = max(v[5], o2);
  }
  if (bad) set_status(status, BH_ERR_NONFINITE);
  int s0 = __shfl_sync(kFull, my_sys, 0);
  bool uniform = __all_sync(kFull, my_sys == s0 || my_sys < 0) && s0 >= 0;
  if (uniform) {
    for (int o = 16; o > 0; o >>= 1)
      for (int a = 0; a < 3; ++a) {
        v[a] = min(v[a], __shfl_xor_sync(kFull, v[a], o));
        v[3 + a] = max(v[3 + a], __shfl_xor_sync(kFull, v[3 + a], o));
      }
    if (lane == 0) {
      for (int a = 0; a < 6; ++a) s_v[warp][a] = v[a];
      s_sys[warp] = s0;
    }
  } else {
    if (my_sys >= 0)
      for (int a = 0; a < 3; ++a) {
        atomicMin(&minmax[6 * my_sys + a], v[a]);
        atomicMax(&minmax[6 * my_sys + 3 + a], v[3 + a]);
      }
    if (lane == 0) s_sys[warp] = -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // merge the warps' partials, one set of atomics per run of equal systems
    int cur = -1;
    unsigned long long acc[6];
    for (int w = 0; w <= kBlock / 32; ++w) {
      int s = (w < kBlock / 32) ? s_sys[w] : -2;
      if (s != cur && cur >= 0) {
        for (int a = 0; a < 3; ++a) {
          atomicMin(&minmax[6 * cur + a], acc[a]);
          atomicMax(&minmax[6 * cur + 3 + a], acc[3 + a]);
        }
        cur = -1;
      }
      if (s >= 0) {
        if (cur < 0) {
          cur = s;
          for (int a = 0; a < 6; ++a) acc[a] = s_v[w][a];
        } else {
          for (int a = 0; a < 3; ++a) {
            acc[a] = min(acc[a], s_v[w][a]);
            acc[3 + a] = max(acc[3 + a], s_v[w][3 + a]);
          }
        }
      }
    }
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    Frame f = {0.0, 0.0, 0.0, 1.0};
    if (offs[s + 1] > offs[s]) {
      double lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = double_of(__ldcg(&minmax[6 * s + a]));
        hi[a] = double_of(__ldcg(&minmax[6 * s + 3 + a]));
      }
      double E = 0.0;
      for (int a = 0; a < 3; ++a) E = fmax(E, __dsub_rn(hi[a], lo[a]));
      double L = 1.0;
      if (E > 0.0) {
        double v2 = __dmul_rn(E, 1.0 + 0x1p-20);
        int e;
        double m = frexp(v2, &e);
        L = (m == 0.5) ? v2 : ldexp(1.0, e);
      }
      f = Frame{lo[0], lo[1], lo[2], L};
    }
    frame[s] = f;
    FrameF ff;
    split2(f.x, ff.ohi[0], ff.olo[0]);
    split2(f.y, ff.ohi[1], ff.olo[1]);
    split2(f.z, ff.ohi[2], ff.olo[2]);
    ff.L = (float)f.w;
    ff.pad = 0.f;
    framef[s] = ff;
  }
  if (threadIdx.x == 0) *ticket = 0;
}

// ----------------------------------------------------------------- keys
// floor(d * 2^k) clamped to [0, qmax], from the bits of d: a product with a
// power of two is exact (or, below 2^-1022, under 1 anyway), so this equals
// clamp(floor(__dmul_rn(d, 2^k))) without FP64 arithmetic.  NaN gives 0.
__device__ __forceinline__ uint32_t quantize(double d, int k, uint32_t qmax) {
  const long long b = __double_as_longlong(d);
  if (b <= 0) return 0;  // negative, -0 or +0
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long frac = (unsigned long long)b & ((1ull << 52) - 1);
  if (e == 0x7ff) return frac ? 0u : qmax;  // NaN, +inf
  // d = m 2^(e' - 1075) with the hidden bit (normal) or e' = 1 (subnormal)
  const unsigned long long m = e ? (frac | (1ull << 52)) : frac;
  const int sh = 1075 - (e ? e : 1) - k;  // d 2^k = m 2^-sh
  if (sh <= 0) return qmax;               // >= 2^52
  if (sh >= 64) return 0;
  const unsigned long long t = m >> sh;
  return t >= qmax ? qmax : (uint32_t)t;
}

// Keys of D levels: q = floor((x - origin) 2^D / L) per axis; the 60-bit word
// interleaves the top 20 bits of q (levels 1..20), the low word (DEEP) the
// remaining D - 20 bits.  DEEP writes both words in input order and the low
// one also into the sort's first buffer.
template <bool FOREST, bool DEEP>
__global__ void __launch_bounds__(kBlock) k_keys(const double *__restrict__ pos, int n,
                                                 const int32_t *__restrict__ offs, int S,
                                                 const Frame *__restrict__ frame, int D, uint64_t *__restrict__ key,
                                                 uint64_t *__restrict__ key_hi0, uint64_t *__restrict__ key_lo0,
                                                 uint32_t *__restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = FOREST ? sys_of(offs, S, i) : 0;
  Frame f = frame[s];
  const int DD = DEEP ? D : kLevels;
  // scale = 2^D / L = 2^k exactly (L is a power of two, possibly subnormal)
  const unsigned long long lb = (unsigned long long)__double_as_longlong(f.w);
  const int le = (int)((lb >> 52) & 0x7ffull);
  const int k = DD - (le ? le - 1023 : -1074 + (63 - __clzll((long long)lb)));
  double o[3] = {f.x, f.y, f.z};
  uint32_t q[3];
  const uint32_t qmax = (1u << DD) - 1u;
  for (int a = 0; a < 3; ++a) q[a] = quantize(__dsub_rn(pos[3 * (size_t)i + a], o[a]), k, qmax);
  if (!DEEP) {
    key[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  } else {
    const int sl = DD - kLevels;
    const uint32_t ml = (1u << sl) - 1u;
    const uint64_t hi = spread3(q[0] >> sl) | (spread3(q[1] >> sl) << 1) | (spread3(q[2] >> sl) << 2);
    const uint64_t lo = spread3(q[0] & ml) | (spread3(q[1] & ml) << 1) | (spread3(q[2] & ml) << 2);
    key_hi0[i] = hi;
    key_lo0[i] = lo;
    key[i] = lo;
  }
  idx[i] = (uint32_t)i;
}

// ----------------------------------------------------------------- sort
constexpr int kSortThreads = 256;  // threads of a digit pass (the first 256 also own one digit each)
constexpr int kSortBlocksPerSm = 2;  // resident blocks of the persistent pass
constexpr int kSortIpt = 16;
constexpr int kSortTile = kSortThreads * kSortIpt;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kValMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookback = 8;  // predecessor tiles read per look-back step
// two tile buffers (8-byte keys, 4-byte indices) and one digit byte per key
constexpr size_t kSortDynSmem = (size_t)kSortTile * (2 * (8 + 4) + 1);

// Digit of a pass: byte `byte` of the key word, or (byte < 0) byte -1 - byte
// of the body's system id.
__device__ __forceinline__ uint32_t sort_digit(uint64_t k, uint32_t v, int byte, const int32_t *offs, int S) {
  if (byte >= 0) return (uint32_t)(k >> (8 * byte)) & 0xffu;
  return ((uint32_t)sys_of(offs, S, (int)v) >> (8 * (-1 - byte))) & 0xffu;
}

// Byte of pass p: passes 0..lo_passes-1 take the low key word, the next 8 the
// 60-bit word, the rest the system id.
__host__ __device__ __forceinline__ int pass_byte(int p, int lo_passes) {
  if (p < lo_passes) return p;
  if (p < lo_passes + 8) return p - lo_passes;
  return -1 - (p - lo_passes - 8);
}

// All digit histograms in one read of the key words (a histogram does not
// depend on the order, so both words are read in input order).
__global__ void __launch_bounds__(kBlock) k_sort_hist(const uint64_t *__restrict__ klo,
                                                      const uint64_t *__restrict__ khi, int n, int lo_passes,
                                                      int passes, const int32_t *__restrict__ offs, int S,
                                                      uint32_t *hist) {
  extern __shared__ uint32_t s_h[];  // [passes][256]
  for (int t = threadIdx.x; t < passes * 256; t += blockDim.x) s_h[t] = 0;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint64_t h = khi[i], l = lo_passes ? klo[i] : 0;
    for (int p = 0; p < passes; ++p)
      atomicAdd(&s_h[p * 256 + sort_digit(p < lo_passes ? l : h, (uint32_t)i, pass_byte(p, lo_passes), offs, S)], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < passes * 256; t += blockDim.x)
    if (s_h[t]) atomicAdd(&hist[t], s_h[t]);
}

// Exclusive prefix of each pass's 256 bins (one block per pass).
__global__ void k_sort_binscan(uint32_t *hist) {
  __shared__ uint32_t s[256];
  uint32_t *h = hist + blockIdx.x * 256;
  s[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int d = 0; d < 256; ++d) {
      uint32_t c = s[d];
      s[d] = acc;
      acc += c;
    }
  }
  __syncthreads();
  h[threadIdx.x] = s[threadIdx.x];
}

// Exclusive scan of the 256 digit values held by threads 0..255 (the other
// threads pass 0 and take part only in the barriers); returns the exclusive
// prefix of v.
__device__ __forceinline__ uint32_t digit_exclusive(uint32_t v, uint32_t *s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31 && warp < 8) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < 8) ? s_warp[lane] : 0;
    for (int o = 1; o < 8; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < 8) s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t before = (warp > 0 && warp < 8) ? s_warp[warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// Asynchronous 16-byte copy global -> shared (cp.async, L2 only); bytes < 16
// reads that many and fills the rest of the 16 with zeros.
__device__ __forceinline__ void copy16_async(void *dst_smem, const void *src, uint32_t bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void copy_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// waits until at most one committed group of this thread is still in flight
__device__ __forceinline__ void copy_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Starts the copy of tile `tile`'s keys and indices into a shared buffer:
// 16-byte pieces, the ones past n zero-filled (their addresses stay inside
// the arrays: a piece with no byte to read points at the array's start).
__device__ __forceinline__ void sort_tile_fetch(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                int n, uint32_t tile, uint64_t *s_kb, uint32_t *s_vb) {
  const int64_t base = (int64_t)tile * kSortTile;
  for (int c = threadIdx.x; c < kSortTile / 2; c += kSortThreads) {  // two keys per piece
    const int64_t e = base + 2 * c;
    const int64_t left = (int64_t)n - e;
    const uint32_t bytes = left >= 2 ? 16u : (left == 1 ? 8u : 0u);
    copy16_async(s_kb + 2 * c, bytes ? (const void *)(kin + e) : (const void *)kin, bytes);
  }
  for (int c = threadIdx.x; c < kSortTile / 4; c += kSortThreads) {  // four indices per piece
    const int64_t e = base + 4 * c;
    const int64_t left = (int64_t)n - e;
    const uint32_t bytes = left >= 4 ? 16u : (left > 0 ? (uint32_t)left * 4u : 0u);
    copy16_async(s_vb + 4 * c, bytes ? (const void *)(vin + e) : (const void *)vin, bytes);
  }
}

// One stable digit pass over `tiles` tiles of kSortTile keys.  A persistent
// block takes tiles in order from a counter (every taken tile's predecessors
// were taken earlier, by running blocks, so waiting on them ends) and, before
// working on its tile, takes the next one and starts copying it into its
// second shared buffer, so that the load of one tile overlaps the work on the
// other.  Per tile: rank the keys by digit in each warp, publish the tile's
// digit counts, sum the predecessors' (decoupled look-back, bounded wait),
// then scatter through shared memory.
__global__ void __launch_bounds__(kSortThreads, kSortBlocksPerSm)
    k_sort_pass(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                uint32_t *__restrict__ vout, int n, uint32_t tiles, int byte, const uint32_t *__restrict__ binbase,
                uint32_t *status, uint32_t *tile_ctr, const int32_t *__restrict__ offs, int S, int32_t *err) {
  __shared__ uint32_t s_wcnt[kSortThreads / 32][256];
  __shared__ uint32_t s_tstart[256];
  __shared__ uint32_t s_gbase[256];
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_tile;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  // two tile buffers (keys, then indices) and the digits of the scatter
  uint64_t *s_kb0 = reinterpret_cast<uint64_t *>(s_dyn);
  uint32_t *s_vb0 = reinterpret_cast<uint32_t *>(s_kb0 + kSortTile);
  uint64_t *s_kb1 = reinterpret_cast<uint64_t *>(s_vb0 + kSortTile);
  uint32_t *s_vb1 = reinterpret_cast<uint32_t *>(s_kb1 + kSortTile);
  uint8_t *s_d = reinterpret_cast<uint8_t *>(s_vb1 + kSortTile);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  uint32_t tile = s_tile;
  if (tile < tiles) sort_tile_fetch(kin, vin, n, tile, s_kb0, s_vb0);
  copy_async_commit();
  int buf = 0;
  while (tile < tiles) {
    uint64_t *s_kb = buf ? s_kb1 : s_kb0;
    uint32_t *s_vb = buf ? s_vb1 : s_vb0;
    __syncthreads();  // everyone has read s_tile and is done with the other buffer
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int t = threadIdx.x; t < (kSortThreads / 32) * 256; t += kSortThreads) (&s_wcnt[0][0])[t] = 0;
    __syncthreads();
    const uint32_t next = s_tile;
    if (next < tiles) sort_tile_fetch(kin, vin, n, next, buf ? s_kb0 : s_kb1, buf ? s_vb0 : s_vb1);
    copy_async_commit();
    copy_async_wait_one();  // this thread's pieces of the current tile have landed
    __syncthreads();        // and everyone's
    const int base = (int)tile * kSortTile;
    const int tile_n = min(kSortTile, n - base);

    uint64_t k[kSortIpt];
    uint32_t v[kSortIpt], d[kSortIpt], r[kSortIpt];
#pragma unroll
    for (int j = 0; j < kSortIpt; ++j) {
      const int le = warp * 32 * kSortIpt + j * 32 + lane;
      const bool ok = le < tile_n;
      k[j] = s_kb[le];
      v[j] = s_vb[le];
      d[j] = ok ? sort_digit(k[j], v[j], byte, offs, S) : 256u;
    }
#pragma unroll
    for (int j = 0; j < kSortIpt; ++j) {
      unsigned peers = __match_any_sync(kFull, d[j]);
      uint32_t cnt = (d[j] < 256) ? s_wcnt[warp][d[j]] : 0;
      r[j] = cnt + __popc(peers & lt);
      __syncwarp();
      if (d[j] < 256 && (peers & lt) == 0) s_wcnt[warp][d[j]] = cnt + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // digit t (threads 0..255): per-warp exclusive offsets and the tile's count
    const int t = threadIdx.x;
    const bool dig = t < 256;
    uint32_t tot = 0;
    if (dig)
      for (int w = 0; w < kSortThreads / 32; ++w) {
        uint32_t c = s_wcnt[w][t];
        s_wcnt[w][t] = tot;
        tot += c;
      }
    uint32_t *my = status + (size_t)tile * 256;
    if (dig) atomicExch(&my[t], (tile == 0 ? kFlagInc : kFlagAgg) | tot);
    uint32_t tstart = digit_exclusive(dig ? tot : 0u, s_scan);
    if (dig) {
      s_tstart[t] = tstart;
      uint32_t excl = 0;
      if (tile > 0) {
        // decoupled look-back, kLookback predecessors per step: their status
        // words are loaded together, then summed from the nearest back to the
        // first inclusive prefix; an unpublished one stops the step and is
        // polled again (tile 0 is always inclusive, so the walk ends)
        int pr = (int)tile - 1;
        int spins = 0;
        while (pr >= 0) {
          uint32_t w[kLookback];
#pragma unroll
          for (int q = 0; q < kLookback; ++q)
            w[q] = (pr - q >= 0) ? __ldcv(&status[(size_t)(pr - q) * 256 + t]) : kFlagInc;
          int q = 0;
          bool found = false;
          for (; q < kLookback; ++q) {
            const uint32_t f = w[q] & ~kValMask;
            if (f == 0) break;
            excl += w[q] & kValMask;
            if (f == kFlagInc) {
              found = true;
              break;
            }
          }
          if (found) break;
          if (q == 0) {
            if (++spins > kSpinLimit) {
              set_status(err, BH_ERR_TIMEOUT);
              break;
            }
            __nanosleep(32);
          }
          pr -= q;
        }
        atomicExch(&my[t], kFlagInc | (excl + tot));
      }
      s_gbase[t] = binbase[t] + excl;
    }
    __syncthreads();
    // scatter into the tile's own buffer (its keys are in registers now) in
    // (digit, arrival) order
#pragma unroll
    for (int j = 0; j < kSortIpt; ++j) {
      if (d[j] < 256) {
        uint32_t lp = s_tstart[d[j]] + s_wcnt[warp][d[j]] + r[j];
        s_kb[lp] = k[j];
        s_vb[lp] = v[j];
        s_d[lp] = (uint8_t)d[j];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile_n; e += kSortThreads) {
      uint32_t dd = s_d[e];
      uint32_t g = s_gbase[dd] + ((uint32_t)e - s_tstart[dd]);
      kout[g] = s_kb[e];
      vout[g] = s_vb[e];
    }
    tile = next;
    buf ^= 1;
  }
}

// dst[j] = src[idx[j]]: a key word in the order of the index array.
__global__ void __launch_bounds__(kBlock) k_gather_key(const uint32_t *__restrict__ idx,
                                                       const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                                       int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) dst[j] = src[idx[j]];
}

// The failure path of the sort's look-back, run on purpose: each thread polls
// kLookback status words of a tile table that nothing publishes, the way a
// tile polls its predecessors, and gives up after `limit` polls without
// progress, latching BH_ERR_TIMEOUT (the context stays usable).
__global__ void __launch_bounds__(kBlock) k_wait_probe(const uint32_t *status, int limit, int32_t *err) {
  const int t = threadIdx.x;
  int spins = 0;
  while (true) {
    uint32_t w[kLookback];
#pragma unroll
    for (int q = 0; q < kLookback; ++q) w[q] = __ldcv(&status[(size_t)q * 256 + t]);
    int q = 0;
    while (q < kLookback && (w[q] & ~kValMask) != 0) ++q;
    if (q == kLookback) return;  // (never: nothing publishes)
    if (++spins > limit) {
      set_status(err, BH_ERR_TIMEOUT);
      return;
    }
    __nanosleep(32);
  }
}

// ----------------------------------------------------------------- move
__global__ void __launch_bounds__(kBlock) k_move(const double *__restrict__ pos, const double *__restrict__ mass,
                                                 const uint32_t *__restrict__ perm, int n, float4 *part_hi,
                                                 float4 *part_lo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  size_t j = perm[i];
  float h[3], l[3];
  for (int a = 0; a < 3; ++a) split2(pos[3 * j + a], h[a], l[a]);
  part_hi[i] = make_float4(h[0], h[1], h[2], (float)mass[j]);
  part_lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// Gather of the integrator state into the new key order (+ the two-float bodies).
__global__ void __launch_bounds__(kBlock) k_move_state(const uint32_t *__restrict__ perm, int n,
                                                       const double *__restrict__ x0, const double *__restrict__ v0,
                                                       const double *__restrict__ m0, const float4 *__restrict__ a0,
                                                       const int32_t *__restrict__ id0, double *x1, double *v1,
                                                       double *m1, float4 *a1, int32_t *id1, float4 *part_hi,
                                                       float4 *part_lo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  size_t j = perm[i];
  float h[3], l[3];
  for (int a = 0; a < 3; ++a) {
    double x = x0[3 * j + a];
    x1[3 * (size_t)i + a] = x;
    v1[3 * (size_t)i + a] = v0[3 * j + a];
    split2(x, h[a], l[a]);
  }
  double m = m0[j];
  m1[i] = m;
  a1[i] = a0[j];
  id1[i] = id0[j];
  part_hi[i] = make_float4(h[0], h[1], h[2], (float)m);
  part_lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// ---------------------------------------------------------------- cells
constexpr int kHalo = kMaxCrit;  // >= N_crit >= N_leaf
// bodies per thread of the level pass (deeper keys carry a second key word
// in shared memory: half as many, to stay within 48 KB of static memory)
template <bool DEEP>
__host__ __device__ constexpr int lv_ipt() {
  return DEEP ? 4 : 8;
}

// Transpose of the warp's 32 x 32 bit matrix whose row r is lane r's word:
// returns column `lane` (bit r = bit `lane` of lane r's word).  Five rounds
// swap the off-diagonal blocks of halves, quarters, ... with xor shuffles.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane) {
  const unsigned m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
  int j = 16;
#pragma unroll
  for (int i = 0; i < 5; ++i, j >>= 1) {
    const unsigned y = __shfl_xor_sync(kFull, x, j);
    x = (lane & j) ? ((x & ~m[i]) | ((y >> j) & m[i])) : ((x & m[i]) | ((y << j) & ~m[i]));
  }
  return x;
}

// Per body: first level it starts a cell at (common prefix with the previous
// key + 1), its leaf level, whether it starts a group; per warp: how many
// cells it starts at each level and how many groups.  DEEP: keys of D > 20
// levels, the low words in skey_lo.
template <bool FOREST, bool DEEP>
__global__ void __launch_bounds__(kBlock) k_levels(const uint64_t *__restrict__ skey,
                                                   const uint64_t *__restrict__ skey_lo, int D, int n,
                                                   const int32_t *__restrict__ offs, int S, int n_leaf, int n_crit,
                                                   uint8_t *lohi, uint8_t *gstart, uint32_t *rowcnt, int W) {
  const int DD = DEEP ? D : kLevels;
  constexpr int kLvIpt = lv_ipt<DEEP>(), kLvTile = kBlock * kLvIpt;
  __shared__ uint64_t s_key[kLvTile + 2 * kHalo];
  __shared__ uint64_t s_klo[DEEP ? kLvTile + 2 * kHalo : 1];
  // common prefix (levels) of the keys at shared positions a and b
  auto lcp = [&](int a, int b) -> int {
    return DEEP ? key_lcp2(s_key[a], s_klo[a], s_key[b], s_klo[b], DD) : key_lcp(s_key[a], s_key[b]);
  };
  __shared__ int8_t s_wl[kLvTile + kHalo];  // lcp of windows of N_leaf + 1 keys starting at b0 - kHalo + t
  __shared__ int8_t s_wc[kLvTile + kHalo];  // lcp of windows of N_crit + 1 keys
  __shared__ int8_t s_tl[kLvTile + kHalo], s_tc[kLvTile + kHalo];  // doubling buffers
  const int b0 = blockIdx.x * kLvTile;
  for (int t = threadIdx.x; t < kLvTile + 2 * kHalo; t += kBlock) {
    int i = b0 - kHalo + t;
    s_key[t] = (i >= 0 && i < n) ? skey[i] : 0;
    if (DEEP) s_klo[t] = (i >= 0 && i < n) ? skey_lo[i] : 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kLvTile + kHalo; t += kBlock) {
    int s0 = b0 - kHalo + t;  // window start
    int8_t wl = -1, wc = -1;
    if (s0 >= 0 && s0 < n) {
      int sb = 0, se = n;
      if (FOREST) {
        int s = sys_of(offs, S, s0);
        sb = offs[s];
        se = offs[s + 1];
      }
      (void)sb;
      if (s0 + n_leaf < se) wl = (int8_t)lcp(t, t + n_leaf);
      if (s0 + n_crit < se) wc = (int8_t)lcp(t, t + n_crit);
    }
    s_wl[t] = wl;
    s_wc[t] = wc;
  }
  __syncthreads();
  // the largest lcp over the N + 1 windows holding a body is a sliding maximum
  // of fixed length: one sparse-table level T[x] = max(w[x .. x + 2^j - 1]),
  // j = floor(log2(N + 1)), built by j doublings, answers it with two reads
  const int len = kLvTile + kHalo;
  const int jl = 31 - __clz(n_leaf + 1), jc = 31 - __clz(n_crit + 1);
  int8_t *al = s_wl, *bl = s_tl, *ac = s_wc, *bc = s_tc;
  for (int m = 0; m < max(jl, jc); ++m) {
    const int d = 1 << m;
    for (int t = threadIdx.x; t < len; t += kBlock) {
      if (m < jl) bl[t] = (int8_t)max((int)al[t], (t + d < len) ? (int)al[t + d] : -1);
      if (m < jc) bc[t] = (int8_t)max((int)ac[t], (t + d < len) ? (int)ac[t + d] : -1);
    }
    __syncthreads();
    if (m < jl) {
      int8_t *x = al;
      al = bl;
      bl = x;
    }
    if (m < jc) {
      int8_t *x = ac;
      ac = bc;
      bc = x;
    }
  }
  // each thread takes bodies j kBlock + threadIdx.x, j < kLvIpt: a warp holds 32
  // consecutive bodies, the unit of the per-warp counts
  for (int j = 0; j < kLvIpt; ++j) {
    const int i = b0 + j * kBlock + threadIdx.x;
    const bool ok = i < n;
    int lo = 1, hi = 0, gs = 0;
    if (ok) {
      int sb = 0;
      if (FOREST) sb = offs[sys_of(offs, S, i)];
      const int t = j * kBlock + threadIdx.x + kHalo;  // position of i in s_key
      int prev = (i > sb) ? lcp(t - 1, t) : -1;
      // windows of N+1 keys starting at i-N .. i (a window's lcp is -1 where it
      // leaves the system, so windows starting before the system's first body count nothing)
      const int wl = max((int)al[t - n_leaf], (int)al[t + 1 - (1 << jl)]);
      const int wc = max((int)ac[t - n_crit], (int)ac[t + 1 - (1 << jc)]);
      int lam = min(wl + 1, DD);
      int mu = wc + 1;  // D + 1: even the level-D cell holds more than N_crit bodies
      lo = prev + 1;
      hi = lam;
      if (mu <= lam) {
        gs = (lo <= mu);
      } else {
        // chunks of N_crit inside a level-D leaf: find the start of the run of equal keys
        const uint64_t kk = s_key[t], kl = DEEP ? s_klo[t] : 0;
        int a = sb, b = i;  // first index in [a, b] with key == (kk, kl)
        while (a < b) {
          int mid = (a + b) >> 1;
          const uint64_t h = skey[mid];
          if (h < kk || (DEEP && h == kk && skey_lo[mid] < kl)) a = mid + 1; else b = mid;
        }
        gs = ((i - a) % n_crit) == 0;
      }
      lohi[2 * (size_t)i] = (uint8_t)lo;
      lohi[2 * (size_t)i + 1] = (uint8_t)hi;
      gstart[i] = (uint8_t)gs;
    }
    const int lane = threadIdx.x & 31;
    const int w = i >> 5;
    // the levels this body starts a cell at, bits lo..hi (hi <= 30); the
    // warp's 32 such words transposed give lane k the bodies starting a cell
    // at level k
    const unsigned levels = (ok && lo <= hi) ? ((2u << hi) - (1u << lo)) : 0u;
    uint32_t mine = (uint32_t)__popc(warp_transpose32(levels, lane));
    unsigned bg = __ballot_sync(kFull, ok && gs);
    if (lane == DD + 1) mine = __popc(bg);  // rows 0..D: cells per level; row D + 1: groups
    if (lane < DD + 2 && w < W) rowcnt[(size_t)lane * W + w] = mine;
  }
}

// Writes every cell (level, leaf flag, first body, parent/first child where
// the same body starts both) and every group start.
template <bool FOREST, bool DEEP>
__global__ void __launch_bounds__(kBlock) k_emit(int n, int D, const int32_t *__restrict__ offs, int S,
                                                 const uint8_t *__restrict__ lohi, const uint8_t *__restrict__ gstart,
                                                 const uint32_t *__restrict__ rowoff, int W,
                                                 const uint64_t *__restrict__ scan_total, int32_t *c_level,
                                                 int32_t *c_pbeg, int32_t *c_parent, int32_t *c_first,
                                                 int32_t *sys_root, int32_t *g_beg, int32_t *g_sys,
                                                 int32_t *counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = i >> 5;
  const bool ok = i < n;
  const unsigned lt = lanemask_lt();
  int lo = 1, hi = 0, gs = 0, s = 0;
  if (ok) {
    lo = lohi[2 * (size_t)i];
    hi = lohi[2 * (size_t)i + 1];
    gs = gstart[i];
    if (FOREST) s = sys_of(offs, S, i);
  }
  const int DD = DEEP ? D : kLevels;
  const uint32_t C = rowoff[(size_t)(DD + 1) * W];
  // this warp's offset in every row (levels 0..D, then groups: at most 32
  // rows), lane r holding row r, all loaded at once
  const int lane = threadIdx.x & 31;
  const uint32_t myoff = (lane <= DD + 1 && w < W) ? rowoff[(size_t)lane * W + w] : 0u;
  // the levels at which some lane of this warp starts a cell
  const bool starts = ok && lo <= hi;
  const int kmin = __reduce_min_sync(kFull, starts ? lo : DD + 1);
  const int kmax = __reduce_max_sync(kFull, starts ? hi : -1);
  int prev = -1;
  unsigned pb = 0;  // which lanes started a cell one level up (none below kmin)
  // this warp's offset one level up
  uint32_t poff = (kmin >= 1 && kmin <= DD) ? __shfl_sync(kFull, myoff, kmin - 1) : 0u;
  for (int k = kmin; k <= kmax; ++k) {
    bool in = ok && lo <= k && k <= hi;
    unsigned b = __ballot_sync(kFull, in);
    const uint32_t off = __shfl_sync(kFull, myoff, k);
    if (in) {
      int cell = (int)(off + __popc(b & lt));
      bool leaf = (k == hi);
      c_level[cell] = k | (leaf ? 32 : 0);
      c_pbeg[cell] = i;
      // parent: the cell this body started one level up, or else the last
      // level-(k-1) cell started before this body (the one holding it, as
      // cells of a level are in body order and nest): the last such start
      // in this warp's lower lanes, or the last one of the earlier warps
      int par = -1;
      if (k > lo) par = prev;
      else if (k > 0) par = (int)(poff + __popc(pb & lt)) - 1;
      c_parent[cell] = par;
      c_first[cell] = -1;
      if (k > lo) c_first[prev] = cell;
      if (k == 0) sys_root[s] = cell;
      prev = cell;
    }
    pb = b;
    poff = off;
  }
  unsigned bg = __ballot_sync(kFull, ok && gs);
  const uint32_t goff = __shfl_sync(kFull, myoff, DD + 1);
  if (ok && gs) {
    int g = (int)(goff - C + __popc(bg & lt));
    g_beg[g] = i;
    g_sys[g] = s;
  }
  if (i == 0) {
    uint32_t G = (uint32_t)(*scan_total) - C;
    counts[0] = (int32_t)C;
    counts[1] = (int32_t)G;
    g_beg[G] = n;
  }
}

// One thread per cell: body range end (galloping search in the sorted keys)
// and, for a leaf, its link word.  A node's children are the cells one
// level down with it as parent, consecutive; the last of them writes the
// node's child count and link word.
template <bool FOREST, bool DEEP>
__global__ void __launch_bounds__(kBlock) k_link(int n, const uint64_t *__restrict__ skey,
                                                 const uint64_t *__restrict__ skey_lo, int D,
                                                 const int32_t *__restrict__ offs, int S,
                                                 const int32_t *__restrict__ counts,
                                                 const int32_t *__restrict__ c_level,
                                                 const int32_t *__restrict__ c_pbeg, int32_t *c_pend,
                                                 const int32_t *__restrict__ c_parent,
                                                 const int32_t *__restrict__ c_first, int32_t *c_nch, int2 *c_link) {
  const int C = counts[0];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    const int lv = c_level[c];
    const int k = lv & 31;
    const bool leaf = lv & 32;
    const int i = c_pbeg[c];
    int se = n;
    if (FOREST) se = offs[sys_of(offs, S, i) + 1];
    int pend = se;
    if (k > 0) {
      // does body j share body i's level-k prefix?
      const bool low = DEEP && k > kLevels;  // the prefix reaches into the low word
      const int sh = low ? 3 * (D - k) : 60 - 3 * k;
      const uint64_t P = low ? skey_lo[i] >> sh : skey[i] >> sh, H = skey[i];
      auto same = [&](int j) -> bool {
        return low ? (skey[j] == H && (skey_lo[j] >> sh) == P) : (skey[j] >> sh) == P;
      };
      int in_run = i, step = 1;
      while (i + step < se && same(i + step)) {
        in_run = i + step;
        step <<= 1;
      }
      int a = in_run + 1, b = min(i + step, se);  // first index with another prefix lies in [a, b]
      while (a < b) {
        int mid = (a + b) >> 1;
        if (same(mid)) a = mid + 1; else b = mid;
      }
      pend = a;
    }
    c_pend[c] = pend;
    if (leaf) {
      c_nch[c] = 0;
      c_link[c] = make_int2(i, (int)((unsigned)(pend - i) | 0x80000000u));
    }
    if (k > 0) {
      const int par = c_parent[c];
      if (c + 1 >= C || c_parent[c + 1] != par) {
        const int f = c_first[par], nch = c - f + 1;
        c_nch[par] = nch;
        c_link[par] = make_int2(f, nch);
      }
    }
  }
}

// ----------------------------------------------------------------- scan
constexpr int kScanIpt = 16;
constexpr int kScanTile = kBlock * kScanIpt;

// Block sums are exact 64-bit sums (a tile of 4096 values below 2^32 sums
// below 2^44), so the total is exact; the scanned values themselves wrap
// modulo 2^32, the width of the output.
__global__ void __launch_bounds__(kBlock) k_scan_up(const uint32_t *__restrict__ in, int64_t n, uint64_t *blocks) {
  __shared__ uint64_t s_w[kBlock / 32];
  const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
  uint64_t sum = 0;
  for (int j = 0; j < kScanIpt; ++j) {
    int64_t i = b0 + j * kBlock + threadIdx.x;
    if (i < n) sum += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kBlock / 32; ++w) t += s_w[w];
    blocks[blockIdx.x] = t;
  }
}

// Exclusive scan of the nb block sums in place, in 64 bits; *total = their sum.
__global__ void __launch_bounds__(1024) k_scan_mid(uint64_t *blocks, int nb, uint64_t *total) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    uint64_t v = (i < nb) ? blocks[i] : 0;
    uint64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = s_w[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    uint64_t carry = s_carry;
    uint64_t excl = carry + (warp ? s_w[warp - 1] : 0) + x - v;
    if (i < nb) blocks[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

__global__ void __launch_bounds__(kBlock) k_scan_down(const uint32_t *__restrict__ in, int64_t n,
                                                      const uint64_t *__restrict__ blocks, uint32_t *out) {
  __shared__ uint32_t s[kScanTile];
  __shared__ uint32_t s_w[kBlock / 32];
  const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
  for (int j = 0; j < kScanIpt; ++j) {
    int64_t i = b0 + j * kBlock + threadIdx.x;
    s[j * kBlock + threadIdx.x] = (i < n) ? in[i] : 0;
  }
  __syncthreads();
  uint32_t loc[kScanIpt];
  uint32_t sum = 0;
  for (int j = 0; j < kScanIpt; ++j) {
    loc[j] = sum;
    sum += s[threadIdx.x * kScanIpt + j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint32_t wb = 0;
  for (int w = 0; w < warp; ++w) wb += s_w[w];
  const uint32_t base = (uint32_t)blocks[blockIdx.x] + wb + x - sum;
  __syncthreads();
  for (int j = 0; j < kScanIpt; ++j) s[threadIdx.x * kScanIpt + j] = base + loc[j];
  __syncthreads();
  for (int j = 0; j < kScanIpt; ++j) {
    int64_t i = b0 + j * kBlock + threadIdx.x;
    if (i < n) out[i] = s[j * kBlock + threadIdx.x];
  }
}

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

// =================================================================== launches
cudaError_t launch_reset(Ctx &c, cudaStream_t s) {
  int n = 6 * c.n_sys;
  k_reset<<<cdiv(n, kBlock), kBlock, 0, s>>>(c.minmax, c.n_sys, c.frame_ticket);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_frame_keys(Ctx &c, const double *pos, const double *mass, cudaStream_t s) {
  const int n = (int)c.n;
  const bool forest = c.n_sys > 1;
  int nb = cdiv(n, 4 * kBlock);
  if (forest)
    k_bbox<true><<<nb, kBlock, 0, s>>>(pos, mass, n, c.offs, c.n_sys, c.minmax, c.frame_ticket, c.frame, c.framef,
                                       c.d_status);
  else
    k_bbox<false><<<nb, kBlock, 0, s>>>(pos, mass, n, c.offs, c.n_sys, c.minmax, c.frame_ticket, c.frame,
                                        c.framef, c.d_status);
  const int D = c.levels, kb = cdiv(n, kBlock);
  if (D > kLevels) {
    if (forest)
      k_keys<true, true><<<kb, kBlock, 0, s>>>(pos, n, c.offs, c.n_sys, c.frame, D, c.key[0], c.key_hi0, c.key_lo0,
                                               c.idx[0]);
    else
      k_keys<false, true><<<kb, kBlock, 0, s>>>(pos, n, c.offs, c.n_sys, c.frame, D, c.key[0], c.key_hi0, c.key_lo0,
                                                c.idx[0]);
  } else {
    if (forest)
      k_keys<true, false><<<kb, kBlock, 0, s>>>(pos, n, c.offs, c.n_sys, c.frame, D, c.key[0], nullptr, nullptr,
                                                c.idx[0]);
    else
      k_keys<false, false><<<kb, kBlock, 0, s>>>(pos, n, c.offs, c.n_sys, c.frame, D, c.key[0], nullptr, nullptr,
                                                 c.idx[0]);
  }
  c.launches += 2;
  return cudaGetLastError();
}

static int sort_sys_passes(int S) {
  if (S <= 1) return 0;
  int bits = 0;
  while ((1 << bits) < S) ++bits;
  return (bits + 7) / 8;
}

// Digit passes over the low key word of a D-level key (0 for D = 20).
static int sort_lo_passes(int D) { return D > kLevels ? (3 * (D - kLevels) + 7) / 8 : 0; }

int sort_passes_for(int S, int D) { return sort_lo_passes(D) + 8 + sort_sys_passes(S); }

cudaError_t build_init_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kSortDynSmem);
  if (e) return e;
  // kSortBlocksPerSm persistent blocks per SM: the largest shared-memory carveout
  return cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}
int64_t sort_tiles_for(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

cudaError_t launch_sort(Ctx &c, cudaStream_t s) {
  const int n = (int)c.n;
  const bool deep = c.levels > kLevels;
  const int lo_passes = sort_lo_passes(c.levels);
  const int passes = sort_passes_for(c.n_sys, c.levels);
  const int tiles = cdiv(n, kSortTile);
  cudaError_t e;
  e = cudaMemsetAsync(c.sort_hist, 0, sizeof(uint32_t) * passes * 256, s);
  if (e) return e;
  e = cudaMemsetAsync(c.sort_status, 0, sizeof(uint32_t) * (size_t)passes * tiles * 256, s);
  if (e) return e;
  e = cudaMemsetAsync(c.sort_tile_ctr, 0, sizeof(uint32_t) * passes, s);
  if (e) return e;
  int hb = min(cdiv(n, kBlock), c.num_sms * 8);
  k_sort_hist<<<hb, kBlock, sizeof(uint32_t) * passes * 256, s>>>(deep ? c.key_lo0 : nullptr,
                                                                   deep ? c.key_hi0 : c.key[0], n, lo_passes, passes,
                                                                   c.offs, c.n_sys, c.sort_hist);
  k_sort_binscan<<<passes, 256, 0, s>>>(c.sort_hist);
  const int grid = min(tiles, c.num_sms * kSortBlocksPerSm);
  for (int p = 0; p < passes; ++p) {
    int src = p & 1;
    if (deep && p == lo_passes) {  // sorted by the low word: bring the 60-bit word into this order
      k_gather_key<<<cdiv(n, kBlock), kBlock, 0, s>>>(c.idx[src], c.key_hi0, c.key[src], n);
      c.launches++;
    }
    k_sort_pass<<<grid, kSortThreads, kSortDynSmem, s>>>(c.key[src], c.idx[src], c.key[src ^ 1], c.idx[src ^ 1],
                                                         n, (uint32_t)tiles, pass_byte(p, lo_passes),
                                                         c.sort_hist + p * 256, c.sort_status + (size_t)p * tiles * 256,
                                                         c.sort_tile_ctr + p, c.offs, c.n_sys, c.d_status);
  }
  c.launches += 2 + passes;
  if (passes & 1) {  // 9 passes (forest of 2..256 systems): bring the result back to buffer 0
    e = cudaMemcpyAsync(c.key[0], c.key[1], sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e) return e;
    e = cudaMemcpyAsync(c.idx[0], c.idx[1], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e) return e;
  }
  if (deep) {  // the low words in the final order
    k_gather_key<<<cdiv(n, kBlock), kBlock, 0, s>>>(c.idx[0], c.key_lo0, c.skey_lo, n);
    c.launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_wait_probe(Ctx &c, int limit, cudaStream_t s) {
  // a tile table of kLookback tiles, all unpublished
  cudaError_t e = cudaMemsetAsync(c.sort_status, 0, sizeof(uint32_t) * kLookback * 256, s);
  if (e) return e;
  k_wait_probe<<<1, kBlock, 0, s>>>(c.sort_status, limit < 1 ? 1 : min(limit, kSpinLimit), c.d_status);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_move(Ctx &c, const double *pos, const double *mass, cudaStream_t s) {
  const int n = (int)c.n;
  k_move<<<cdiv(n, kBlock), kBlock, 0, s>>>(pos, mass, c.idx[0], n, c.part_hi, c.part_lo);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_move_state(Ctx &c, cudaStream_t s) {
  const int n = (int)c.n;
  const int a = c.state_cur, b = a ^ 1;
  k_move_state<<<cdiv(n, kBlock), kBlock, 0, s>>>(c.idx[0], n, c.st_x[a], c.st_v[a], c.st_m[a], c.st_a[a],
                                                  c.st_id[a], c.st_x[b], c.st_v[b], c.st_m[b], c.st_a[b],
                                                  c.st_id[b], c.part_hi, c.part_lo);
  c.state_cur = b;
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_scan_u32(Ctx &c, const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
  int nb = cdiv(n, kScanTile);
  if (nb == 0) {
    c.launches++;
    return cudaMemsetAsync(c.scan_total, 0, sizeof(uint64_t), s);
  }
  k_scan_up<<<nb, kBlock, 0, s>>>(in, n, c.scan_blocks);
  k_scan_mid<<<1, 1024, 0, s>>>(c.scan_blocks, nb, c.scan_total);
  k_scan_down<<<nb, kBlock, 0, s>>>(in, n, c.scan_blocks, out);
  c.launches += 3;
  return cudaGetLastError();
}

// The same three scan kernels with caller-chosen scratch: `blocks` holds
// scan_blocks_for(n) 64-bit block sums, `total` receives the exact sum of all n
// values (out wraps modulo 2^32).
cudaError_t launch_scan_u32_raw(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *blocks, uint64_t *total,
                                cudaStream_t s) {
  int nb = cdiv(n, kScanTile);
  if (nb == 0) return cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
  k_scan_up<<<nb, kBlock, 0, s>>>(in, n, blocks);
  k_scan_mid<<<1, 1024, 0, s>>>(blocks, nb, total);
  k_scan_down<<<nb, kBlock, 0, s>>>(in, n, blocks, out);
  return cudaGetLastError();
}

int64_t scan_blocks_for(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

template <bool FOREST, bool DEEP>
static cudaError_t cells_impl(Ctx &c, cudaStream_t s) {
  const int n = (int)c.n, D = c.levels;
  const int W = cdiv(n, 32);
  const int nb = cdiv(n, kBlock);
  k_levels<FOREST, DEEP><<<cdiv(n, kBlock * lv_ipt<DEEP>()), kBlock, 0, s>>>(
      c.key[0], c.skey_lo, D, n, c.offs, c.n_sys, c.p.n_leaf, c.p.n_crit, c.lohi, c.gstart, c.rowcnt, W);
  c.launches++;
  cudaError_t e = launch_scan_u32(c, c.rowcnt, c.rowoff, (int64_t)(D + 2) * W, s);
  if (e) return e;
  k_emit<FOREST, DEEP><<<nb, kBlock, 0, s>>>(n, D, c.offs, c.n_sys, c.lohi, c.gstart, c.rowoff, W, c.scan_total,
                                             c.c_level, c.c_pbeg, c.c_parent, c.c_first, c.sys_root,
                                             c.g_beg, c.g_sys, c.d_counts);
  k_link<FOREST, DEEP><<<c.num_sms * 8, kBlock, 0, s>>>(n, c.key[0], c.skey_lo, D, c.offs, c.n_sys, c.d_counts,
                                                        c.c_level, c.c_pbeg, c.c_pend, c.c_parent, c.c_first,
                                                        c.c_nch, c.c_link);
  c.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_cells(Ctx &c, cudaStream_t s) {
  const bool forest = c.n_sys > 1, deep = c.levels > kLevels;
  if (forest) return deep ? cells_impl<true, true>(c, s) : cells_impl<true, false>(c, s);
  return deep ? cells_impl<false, true>(c, s) : cells_impl<false, false>(c, s);
}

}  // namespace bh
