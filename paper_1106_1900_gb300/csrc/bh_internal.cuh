// bh_internal.cuh -- context layout, launch entry points and device helpers
// shared by the library's translation units (never by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bh.h"

namespace bh {

constexpr int kLevels = 20;          // the 60-bit key word: levels 1..20 (App. B)
constexpr int kLevelsMax = 30;       // deepest key: 90 bits, a second word for levels 21..30
constexpr int kRowsMax = kLevelsMax + 2;  // cell levels 0..D + one row of group starts (<= 32)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kCostBuckets = 256;  // logarithmic buckets of a group's estimated evaluation cost
constexpr int kMaxCrit = 256;      // largest group size N_crit (the level build's window halo)
constexpr int kPoolAlign = 4;      // split walk: list-pool offsets in units of 4 entries (2^34 entries addressable)

// Frame of one system: origin (per-axis minimum) and power-of-two side L.
struct __align__(32) Frame {
  double x, y, z, w;
};

// The same frame as floats: the origin as two-float pairs (hi + lo = origin to
// ~2^-48) and the side L (a power of two, exact), for FP32-only cell geometry.
struct __align__(32) FrameF {
  float ohi[3], olo[3], L, pad;
};

// ------------------------------------------------------------ context
struct Ctx {
  bh_params p;
  int device = 0;
  int num_sms = 0;
  int64_t n_max = 0;
  int32_t s_max = 1;
  int64_t c_max = 0;   // cell-table bound
  int levels = kLevels;  // key depth D (bh_params.key_levels)
  int trav_grid = 0;   // persistent traversal blocks (split walk)
  int eval_grid = 0;   // persistent evaluation blocks (split walk)
  int walk_grid = 0;   // persistent blocks of the fused walk
  int trav_warps_total = 0;  // warps that own a level stack and list scratch
  int walk_smem = 0;
  int64_t pool_cap = 0;  // interaction-list pool entries
  size_t ws_bytes = 0;
  char *ws = nullptr;

  // sizes of the current tree
  int64_t n = 0;
  int32_t n_sys = 1;
  bool built = false;       // bh_build* done
  bool forces = false;      // bh_compute_forces done since build
  bool have_state = false;  // bh_set_state done
  bool have_acc = false;    // a_old valid for the state
  bool split_open = false;  // bh_step_begin done, bh_step_end not yet
  int split_init = 0;       // ... for the initial force evaluation
  int state_cur = 0;        // which state buffer (0/1) is current
  // block time-steps: levels k (steps dt_max 2^-k) on integer ticks of dt_max 2^-k_max
  bool block_on = false;    // bh_block_start done since the state was loaded
  bool block_tree = false;  // the tree matches the state's body order (a refresh is possible)
  double blk_dt_max = 0.0, blk_tick = 0.0, blk_eta = 0.0;
  int blk_kmax = 0;
  int64_t host_offsets_sig = -1;

  // ---- device buffers (carved from the workspace)
  // per system
  int32_t *offs;                 // [S+1]
  unsigned long long *minmax;    // [S][6] order-preserving bits of min xyz, max xyz
  Frame *frame;                  // [S] origin xyz, L
  FrameF *framef;                // [S] the same as float pairs
  int32_t *sys_root;             // [S]
  uint32_t *frame_ticket;        // [1]
  // per body
  uint64_t *key[2];             // sort ping-pong; key[0] = the sorted 60-bit words (levels 1..20)
  uint32_t *idx[2];
  uint64_t *key_hi0, *key_lo0;   // D > 20: both key words in input order
  uint64_t *skey_lo;             // D > 20: the sorted low words (levels 21..D); else null
  float4 *part_hi, *part_lo;     // sorted bodies: (x_hi, y_hi, z_hi, m), (x_lo, y_lo, z_lo, 0)
  uint8_t *lohi;                 // [n][2] first level started, last level (leaf level)
  uint8_t *gstart;               // [n] group start flag
  float4 *acc_sorted;            // walk output in sorted order (ax, ay, az, phi)
  double *st_x[2], *st_v[2], *st_m[2];
  float4 *st_a[2];
  int32_t *st_id[2];
  int64_t *st_t[2];              // block time-steps: tick of the body's last update
  int32_t *st_k[2];              // block time-steps: the body's level
  double *pred_x;                // [n][3] positions predicted to the block time (state order)
  double *pred_s;                // [n][3] the same after a rebuild's permutation (sorted order)
  uint8_t *g_active;             // [G] group holds a body due at the block time
  unsigned long long *d_block;   // [0] block time (ticks), [1] active bodies, [2] deepest level
  double *h_pos, *h_mass;        // staging for bh_forces_host
  float *h_acc, *h_pot;
  // per warp of the level pass
  uint32_t *rowcnt;              // [D + 2][W]
  uint32_t *rowoff;              // [D + 2][W]
  // per cell
  int32_t *c_level, *c_pbeg, *c_pend, *c_parent, *c_first, *c_nch;
  int2 *c_link;                  // walk link {first, count | leaf << 31}
  float4 *c_mom;                 // [C][4] moments (see k_moments.cu)
  float4 *c_mac;                 // [C] com_hi xyz, l/theta + delta
  float4 *c_mac_lo;              // [C] key depth > 20: the low parts of c_mac's position; else null
  // per group
  int32_t *g_beg;                // [G+1]
  int32_t *g_sys;                // [G]
  int32_t *g_npc, *g_npp;        // [G] list lengths of the last walk
  unsigned long long *g_csum, *g_psum;
  // sort scratch
  uint32_t *sort_hist;           // [passes][256]
  uint32_t *sort_status;         // [passes][tiles][256]
  uint32_t *sort_tile_ctr;       // [passes]
  int sort_max_passes = 0;
  int64_t sort_tiles_max = 0;
  // scan scratch
  uint64_t *scan_blocks;         // [blocks] exact 64-bit block sums of the scan
  uint64_t *scan_total;          // [1]
  // walk
  int32_t *walk_stack;           // [traversal warps][2][stack_capacity]
  int32_t *list_scratch;         // [walking warps][2][list_buffer (fused) or list_capacity (split)]
  float4 *acc_hold;              // [2 N] fused walk: per body (hi, lo) sums between evaluations of a list
  uint32_t *list_pool;           // [pool_cap] every group's cell list then particle list
  unsigned long long *pool_ctr;  // [1]
  int4 *g_list;                  // [G] {pool offset, cells, bodies, estimated evaluation cost}
  uint32_t *work_hist;           // [2][kCostBuckets] groups per cost bucket, placement counters
  int32_t *g_order;              // [G] groups in order of decreasing estimated cost
  uint32_t *walk_queue;          // [2] traversal, evaluation
  // scalars
  int32_t *d_counts;             // [0] C, [1] G, [2] max level, [3] groups in the walk's order
  unsigned long long *d_totals;  // [0] pp, [1] pc, [2] walk launches
  int32_t *d_status;             // [1]
  double *d_diag;                // [5 + blocks*5]

  // host side bookkeeping
  long long launches = 0;
  bool profiling = false;
  bool capturing = false;
  cudaEvent_t ev[BH_NPHASES + 1][2] = {};
  float phase_ms[BH_NPHASES] = {};
  bool phase_rec[BH_NPHASES + 1] = {};
  cudaStream_t cap_stream = nullptr;
  // one captured step per state-buffer parity (the state swaps buffers every step)
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  long long graph_launches[2] = {0, 0};
  double g_dt = 0;
  float g_theta = -1, g_eps = -1;
};

// ------------------------------------------------------------ launches
// k_build.cu
cudaError_t launch_reset(Ctx &c, cudaStream_t s);
cudaError_t launch_frame_keys(Ctx &c, const double *pos, const double *mass, cudaStream_t s);
cudaError_t launch_sort(Ctx &c, cudaStream_t s);  // key[0]/idx[0] -> sorted key[0]/idx[0]
cudaError_t launch_move(Ctx &c, const double *pos, const double *mass, cudaStream_t s);
cudaError_t launch_wait_probe(Ctx &c, int limit, cudaStream_t s);  // failure path of a bounded wait
cudaError_t launch_move_state(Ctx &c, cudaStream_t s);  // gather state cur -> other, fills part_hi/lo
cudaError_t launch_cells(Ctx &c, cudaStream_t s);
cudaError_t launch_scan_u32(Ctx &c, const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s);
cudaError_t launch_scan_u32_raw(const uint32_t *in, uint32_t *out, int64_t n, uint64_t *blocks, uint64_t *total,
                                cudaStream_t s);
int64_t scan_blocks_for(int64_t n);
// k_moments.cu
cudaError_t launch_moments(Ctx &c, cudaStream_t s);
cudaError_t launch_moments_refresh(Ctx &c, cudaStream_t s);
cudaError_t launch_mac(Ctx &c, float theta, cudaStream_t s);
// k_walk.cu
enum OutMode { kOutCaller = 0, kOutSorted = 1 };
cudaError_t launch_walk(Ctx &c, float theta, float eps, OutMode mode, float *acc, float *pot, cudaStream_t s,
                        const uint8_t *g_active = nullptr);
int walk_smem_bytes(int warps);
cudaError_t launch_mark_groups(Ctx &c, int g0, int g1, cudaStream_t s);  // g_active = [g0, g1)
int walk_list_stride(const bh_params &p);  // ints of list scratch per walking warp
void walk_grids(int *trav_blocks_per_sm, int *eval_blocks_per_sm, int *fused_blocks_per_sm);
// the fused walk unless the split form is asked for or the FP64 evaluation needs the pool
inline bool walk_is_fused(const bh_params &p) { return p.walk_split == 0 && p.walk_variant != 2; }
int walk_block_warps();
cudaError_t walk_init_attrs(int smem);
cudaError_t build_init_attrs();
// k_block.cu
cudaError_t launch_block_levels(Ctx &c, double eps, cudaStream_t s);
cudaError_t launch_block_predict(Ctx &c, cudaStream_t s);
cudaError_t launch_move_block(Ctx &c, cudaStream_t s);
cudaError_t launch_block_parts(Ctx &c, cudaStream_t s);
cudaError_t launch_group_active(Ctx &c, cudaStream_t s);
cudaError_t launch_block_correct(Ctx &c, double eps, bool rebuilt, cudaStream_t s);
cudaError_t launch_block_get(Ctx &c, int32_t *level, int64_t *tick, cudaStream_t s);
// k_integrate.cu
cudaError_t launch_predict(Ctx &c, double dt, cudaStream_t s);
cudaError_t launch_correct(Ctx &c, double dt, cudaStream_t s);
cudaError_t launch_load_state(Ctx &c, const double *pos, const double *vel, const double *mass, cudaStream_t s);
cudaError_t launch_get_state(Ctx &c, double *pos, double *vel, float *acc, float *pot, cudaStream_t s);
cudaError_t launch_diag(Ctx &c, cudaStream_t s);
cudaError_t launch_fma_probe(int blocks, int threads, int iters, float *sink, cudaStream_t s);
// k_direct.cu
cudaError_t launch_direct(const double *pos, const double *mass, int n, const int32_t *targets, int nt, float eps,
                          float *acc, float *pot, cudaStream_t s);

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ void set_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Index of the system holding sorted/input position i: last s with offs[s] <= i.
__device__ __forceinline__ int sys_of(const int32_t *offs, int S, int i) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(offs + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Common prefix of two 60-bit keys, in levels (0..20).
__device__ __forceinline__ int key_lcp(uint64_t a, uint64_t b) {
  uint64_t x = a ^ b;
  if (x == 0) return kLevels;
  int h = 63 - __clzll((long long)x);
  return (59 - h) / 3;
}

// Common prefix of two keys of D levels stored as (60-bit word, low word of
// 3 (D - 20) bits), in levels (0..D).
__device__ __forceinline__ int key_lcp2(uint64_t ha, uint64_t la, uint64_t hb, uint64_t lb, int D) {
  if (ha != hb) return key_lcp(ha, hb);
  const uint64_t x = la ^ lb;
  if (x == 0) return D;
  const int h = 63 - __clzll((long long)x);
  return kLevels + (3 * (D - kLevels) - 1 - h) / 3;
}

// Keep the low 20 bits of v, bit b moved to bit 3b (a 60-bit spread).
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0xfffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Inverse of spread3: bits 0, 3, 6, ... of x gathered into the low 20 bits.
__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x00000000001fffffull;
  return (uint32_t)x;
}

// FP32 <-> FP64 conversions on the integer units.  GB300's FP64 pipe runs
// at a small fraction of its FP32 rate and executes the hardware
// conversions too, so the state updates and the two-float splits that
// convert every body's coordinates were bound by it.  Both are written from
// the IEEE 754 binary32 / binary64 formats.
//
// widen: exact.  A normal number keeps sign and mantissa (moved up 29 bits)
// and its biased exponent gains 1023 - 127 = 896; a subnormal m 2^-149 is
// normalised (leading bit p of m: exponent p + 874, mantissa m shifted up
// 23 - p bits); zeros, infinities and NaNs map to their binary64 forms.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint64_t bits = (uint64_t)(u >> 31) << 63;
  if (e == 0xffu) {
    bits |= (0x7ffull << 52) | ((uint64_t)m << 29);
  } else if (e != 0u) {
    bits |= ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m != 0u) {
    const uint32_t p = 31u - (uint32_t)__clz((int)m);
    bits |= ((uint64_t)(p + 874u) << 52) | ((uint64_t)((m << (23u - p)) & 0x7fffffu) << 29);
  }
  return __longlong_as_double((long long)bits);
}

// narrow_rn: round to nearest, ties to even, for results in the normal
// binary32 range (biased exponent 897..1150 of the binary64 input): keep the
// top 23 mantissa bits, and add one unit when the 29 dropped bits exceed
// half a unit or equal it with an odd last bit (a carry steps the exponent,
// to infinity past the largest float).  Zeros keep their sign; every other
// input (subnormal or overflowing results, infinities, NaN) takes the
// hardware conversion.
__device__ __forceinline__ float narrow_rn(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  if (e >= 897u && e <= 1150u) {
    const uint64_t m = b & 0xfffffffffffffull;
    uint32_t r = ((e - 896u) << 23) | (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1fffffffu);
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ++r;
    return __uint_as_float(sign | r);
  }
  if ((b << 1) == 0) return __uint_as_float(sign);
  return __double2float_rn(x);
}

// x = hi + lo: hi the float nearest x, lo the float nearest the exact rest
// x - hi (one FP64 subtraction).
__device__ __forceinline__ void split2(double x, float &hi, float &lo) {
  hi = narrow_rn(x);
  lo = narrow_rn(__dsub_rn(x, widen(hi)));
}

}  // namespace bh
