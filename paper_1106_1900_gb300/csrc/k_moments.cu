// k_moments.cu -- monopole + quadrupole moments of every cell (§3.2, Fig. 4).
//
// The paper computes the leaves in parallel and then the nodes level by
// level, bottom to top, from the moments one level below.  Here too: one
// launch per level, from the deepest up, over that level's contiguous range
// of cells (cells are stored in level order); a leaf from its bodies, a node
// from its children in index order, each in one pass over its records (the
// quadrupole accumulated about the geometric centre, then moved to the
// centre of mass).  Every cell is one thread's work and no thread waits for
// another.
//
// Arithmetic is FP32 in cell-relative coordinates (the paper uses FP64 on
// hardware whose FP32 path lost accuracy in absolute coordinates): a body
// offset from the cell's geometric centre is (x_hi - c_hi) + (x_lo - c_lo)
// from the two-float forms of both; children's centres of mass enter the
// parent through the parallel-axis shift.
//
// Record per cell (4 x float4):
//   mom[4c+0] = (com_hi.x, com_hi.y, com_hi.z, M)
//   mom[4c+1] = (com_lo.x, com_lo.y, com_lo.z, delta = |com - centre|)
//   mom[4c+2] = (Qxx, Qyy, Qzz, Qxy)
//   mom[4c+3] = (Qxz, Qyz, l, 0)         Q = sum m (3 r r^T - r^2 I) about com
#include <cuda_runtime.h>

#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kBlock = 256;
constexpr int kBatch = 4;  // a cell's items (bodies or children) loaded together

struct Centre {
  float hi[3], lo[3];  // geometric centre as a two-float sum (hi + lo to ~2^-48)
  float l;             // side
};

// a + b = s + e exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// s + c += v, the rounding error of s + v kept in c (TwoSum)
__device__ __forceinline__ void add_compensated(float &s, float &c, float v) {
  float t, e;
  two_sum(s, v, t, e);
  s = t;
  c += e;
}

// (hi, lo) -> the same sum with hi the rounded value and |lo| <= ulp(hi)/2
// (TwoSum: exact whatever the magnitudes).  The walk reads the high part alone
// (the opening test), so it must be the correctly rounded value.
__device__ __forceinline__ void renormalise(float &hi, float &lo) {
  float s, e;
  two_sum(hi, lo, s, e);
  hi = s;
  lo = e;
}

// Key words of the sorted bodies: the 60-bit word (levels 1..20) and, for a
// key depth D > 20, the low word (levels 21..D).
struct Keys {
  const uint64_t *__restrict__ hi;
  const uint64_t *__restrict__ lo;
  int D;
};

// Integer corner along axis a of the level-k cell holding sorted body i: the
// top k bits of the body's quantised coordinate (k <= D).
template <bool DEEP>
__device__ __forceinline__ uint32_t cell_corner(const Keys &K, int k, int i, int a) {
  if (k == 0) return 0u;
  const uint32_t top = compact3(K.hi[i] >> a);  // levels 1..20
  if (!DEEP || k <= kLevels) return top >> (kLevels - k);
  return (top << (k - kLevels)) | (compact3(K.lo[i] >> a) >> (K.D - k));
}

// Geometric centre origin + (i + 1/2) l of the level-k cell holding sorted
// body i, l = L 2^-k.  In FP32 when the frame allows: (i + 1/2) l is exact
// (i < 2^23, l a power of two) and TwoSum adds it to the origin's float pair;
// otherwise (a side below 2^-100 or above 2^100, or a cell below level 23 of
// a deeper key) in FP64, where (i + 1/2) l is exact for i < 2^30.
template <bool FOREST, bool DEEP>
__device__ __forceinline__ Centre cell_centre(int k, int i, const Keys &K, const int32_t *__restrict__ offs, int S,
                                              const Frame *__restrict__ frame, const FrameF *__restrict__ framef) {
  const int s = FOREST ? sys_of(offs, S, i) : 0;
  const FrameF f = framef[s];
  Centre C;
  if (f.L > 0x1p-100f && f.L < 0x1p100f && (!DEEP || k <= 23)) {
    const float l = ldexpf(f.L, -k);
    for (int a = 0; a < 3; ++a) {
      const uint32_t corner = cell_corner<DEEP>(K, k, i, a);
      float e;
      two_sum(f.ohi[a], ((float)corner + 0.5f) * l, C.hi[a], e);
      C.lo[a] = e + f.olo[a];
      renormalise(C.hi[a], C.lo[a]);  // the sum may have cancelled: lo is not small then
    }
    C.l = l;
  } else {
    const Frame g = frame[s];
    const double l = ldexp(g.w, -k);
    const double o[3] = {g.x, g.y, g.z};
    for (int a = 0; a < 3; ++a) {
      const uint32_t corner = cell_corner<DEEP>(K, k, i, a);
      split2(__dadd_rn(o[a], __dmul_rn((double)corner + 0.5, l)), C.hi[a], C.lo[a]);
    }
    C.l = (float)l;
  }
  return C;
}

// centre of mass = centre + cm (float offsets), as a two-float sum
__device__ __forceinline__ void write_cell(float4 *mom, int c, const Centre &C, float M, const float cm[3],
                                           const float Q[6], float l) {
  float hi[3], lo[3];
  for (int a = 0; a < 3; ++a) {
    float e;
    two_sum(C.hi[a], cm[a], hi[a], e);
    lo[a] = e + C.lo[a];
    renormalise(hi[a], lo[a]);
  }
  float delta = sqrtf(cm[0] * cm[0] + cm[1] * cm[1] + cm[2] * cm[2]);
  mom[4 * (size_t)c + 0] = make_float4(hi[0], hi[1], hi[2], M);
  mom[4 * (size_t)c + 1] = make_float4(lo[0], lo[1], lo[2], delta);
  mom[4 * (size_t)c + 2] = make_float4(Q[0], Q[1], Q[2], Q[3]);
  mom[4 * (size_t)c + 3] = make_float4(Q[4], Q[5], l, 0.f);
}

__device__ __forceinline__ void add_point_quad(float Q[6], float m, float dx, float dy, float dz) {
  float r2 = dx * dx + dy * dy + dz * dz;
  Q[0] += m * (3.f * dx * dx - r2);
  Q[1] += m * (3.f * dy * dy - r2);
  Q[2] += m * (3.f * dz * dz - r2);
  Q[3] += m * 3.f * dx * dy;
  Q[4] += m * 3.f * dx * dz;
  Q[5] += m * 3.f * dy * dz;
}

// Q about the centre of mass c (offset from the geometric centre) from Q
// about the geometric centre: Q_c = Q_G - M (3 c c^T - |c|^2 I) (the
// parallel-axis rule for a traceless quadrupole; Q_G ~ M l^2, so the
// rounding of the difference stays ~1e-7 M l^2 however small Q_c is).
__device__ __forceinline__ void shift_to_com(float Q[6], float M, const float cm[3]) {
  const float c2 = cm[0] * cm[0] + cm[1] * cm[1] + cm[2] * cm[2];
  Q[0] -= M * (3.f * cm[0] * cm[0] - c2);
  Q[1] -= M * (3.f * cm[1] * cm[1] - c2);
  Q[2] -= M * (3.f * cm[2] * cm[2] - c2);
  Q[3] -= M * 3.f * cm[0] * cm[1];
  Q[4] -= M * 3.f * cm[0] * cm[2];
  Q[5] -= M * 3.f * cm[1] * cm[2];
}

// One cell's moments in one pass over its items: a leaf's bodies (sorted
// range pbeg .. pend) or a node's nch children first .. first + nch - 1 (one
// level deeper, already complete), in index order.  A body is an item of
// mass m at its position with no quadrupole of its own; a child is one of
// mass M at its centre of mass carrying its quadrupole.  Mass and first
// moments are taken about the cell's geometric centre in compensated sums
// (TwoSum: a leaf at the deepest level may hold thousands of bodies, whose
// plain FP32 sum of equal masses drifts by ~n ulp); the quadrupole is summed
// about the geometric centre (the items' own plus the parallel-axis term of
// each item's offset) and moved to the centre of mass at the end.  Items
// are loaded kBatch at a time, the batch's loads issued together.
// REFRESH: the tree is unchanged but its bodies moved (block time-steps); a
// cell keeps its geometric centre and its size grows to the smallest cube
// about that centre holding its bodies (a leaf) or its children's cubes (a
// node, l/2 + the largest child side), never below its built size.
template <bool FOREST, bool REFRESH, bool DEEP>
__device__ __forceinline__ void cell_moments(int c, int k, bool leaf, int pbeg, int pend, int first, int nch,
                                             const Keys &K, const int32_t *__restrict__ offs, int S,
                                             const Frame *__restrict__ frame, const FrameF *__restrict__ framef,
                                             const float4 *__restrict__ part_hi, const float4 *__restrict__ part_lo,
                                             float4 *mom) {
  const Centre G = cell_centre<FOREST, DEEP>(k, pbeg, K, offs, S, frame, framef);
  const int cnt = leaf ? pend - pbeg : nch;
  float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
  float eM = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
  float ext = 0.f, lch = 0.f;
  float Q[6] = {0, 0, 0, 0, 0, 0};
  for (int i0 = 0; i0 < cnt; i0 += kBatch) {
    float4 A[kBatch], B[kBatch], Q0[kBatch], Q1[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      Q0[j] = Q1[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 + j < cnt) {
        if (leaf) {
          A[j] = part_hi[pbeg + i0 + j];
          B[j] = part_lo[pbeg + i0 + j];
        } else {
          const size_t r = 4 * (size_t)(first + i0 + j);
          A[j] = mom[r];
          B[j] = mom[r + 1];
          Q0[j] = mom[r + 2];
          Q1[j] = mom[r + 3];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (i0 + j >= cnt) break;
      const float m = A[j].w;
      const float dx = (A[j].x - G.hi[0]) + (B[j].x - G.lo[0]);
      const float dy = (A[j].y - G.hi[1]) + (B[j].y - G.lo[1]);
      const float dz = (A[j].z - G.hi[2]) + (B[j].z - G.lo[2]);
      if (REFRESH) {
        ext = fmaxf(ext, fmaxf(fabsf(dx), fmaxf(fabsf(dy), fabsf(dz))));
        lch = fmaxf(lch, Q1[j].z);
      }
      add_compensated(M, eM, m);
      add_compensated(sx, ex, m * dx);
      add_compensated(sy, ey, m * dy);
      add_compensated(sz, ez, m * dz);
      Q[0] += Q0[j].x;
      Q[1] += Q0[j].y;
      Q[2] += Q0[j].z;
      Q[3] += Q0[j].w;
      Q[4] += Q1[j].x;
      Q[5] += Q1[j].y;
      add_point_quad(Q, m, dx, dy, dz);
    }
  }
  M += eM;
  sx += ex;
  sy += ey;
  sz += ez;
  float cm[3] = {0.f, 0.f, 0.f};
  if (M > 0.f) {
    cm[0] = sx / M;
    cm[1] = sy / M;
    cm[2] = sz / M;
  }
  shift_to_com(Q, M, cm);
  float l = G.l;
  if (REFRESH) l = leaf ? fmaxf(G.l, 2.f * ext) : fmaxf(G.l, fmaf(0.5f, G.l, lch));
  write_cell(mom, c, G, M, cm, Q, l);
}

// The cells of level k (a contiguous range: cells are in level order, the
// level scan's offsets rowoff[k W] .. rowoff[(k + 1) W]): leaves from their
// bodies, nodes from their children, which the previous launch (level
// k + 1) completed.  Launched for k = D down to 0, so the pass runs bottom
// up level by level, as the paper's, with no waiting and no counters.
template <bool FOREST, bool REFRESH, bool DEEP>
__global__ void __launch_bounds__(kBlock) k_moments_level(const Keys K, const int32_t *__restrict__ offs, int S,
                                                          const Frame *__restrict__ frame,
                                                          const FrameF *__restrict__ framef,
                                                          const uint32_t *__restrict__ rowoff, int W, int k,
                                                          const int32_t *__restrict__ c_level,
                                                          const int32_t *__restrict__ c_pbeg,
                                                          const int32_t *__restrict__ c_pend,
                                                          const int32_t *__restrict__ c_first,
                                                          const int32_t *__restrict__ c_nch,
                                                          const float4 *__restrict__ part_hi,
                                                          const float4 *__restrict__ part_lo, float4 *mom) {
  const int c0 = (int)rowoff[(size_t)k * W], c1 = (int)rowoff[(size_t)(k + 1) * W];
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x) {
    // the cell's table entries, loaded together
    const int lv = c_level[c], pbeg = c_pbeg[c], pend = c_pend[c], first = c_first[c], nch = c_nch[c];
    cell_moments<FOREST, REFRESH, DEEP>(c, lv & 31, (lv & 32) != 0, pbeg, pend, first, min(max(nch, 0), 8), K, offs,
                                        S, frame, framef, part_hi, part_lo, mom);
  }
}

// Opening radius of Eq. 1 for this theta: r_open = l/theta + delta, beside the
// centre of mass (high part) that the walk's opening test reads; with keys
// deeper than 20 levels also the low part (mac_lo non-null), since a cell
// can then be smaller than the float spacing at its position.
__global__ void __launch_bounds__(kBlock) k_mac(const int32_t *__restrict__ counts, const float4 *__restrict__ mom,
                                                float inv_theta, float4 *mac, float4 *mac_lo, uint32_t *queue,
                                                unsigned long long *pool_ctr, uint32_t *work_hist) {
  const int C = counts[0];
  if (blockIdx.x == 0) {  // the walk's group counters, list pool and cost histogram start empty
    if (threadIdx.x == 0) {
      queue[0] = 0;
      queue[1] = 0;
      pool_ctr[0] = 0;
    }
    for (int i = threadIdx.x; i < 2 * kCostBuckets; i += blockDim.x) work_hist[i] = 0;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    float4 a = mom[4 * (size_t)c];
    float4 b = mom[4 * (size_t)c + 1];
    float l = mom[4 * (size_t)c + 3].z;
    mac[c] = make_float4(a.x, a.y, a.z, fmaf(l, inv_theta, b.w));
    if (mac_lo) mac_lo[c] = make_float4(b.x, b.y, b.z, 0.f);
  }
}

// The minimal-distance criterion's record: the cell's geometric centre
// (rounded to float) and its half side l/2 (exact); the walk tests the gap
// between this cube and the group's box against l/theta = (l/2)(2/theta).
template <bool FOREST, bool DEEP>
__global__ void __launch_bounds__(kBlock) k_mac_box(const int32_t *__restrict__ counts, const Keys K,
                                                    const int32_t *__restrict__ offs, int S,
                                                    const Frame *__restrict__ frame,
                                                    const FrameF *__restrict__ framef,
                                                    const int32_t *__restrict__ c_level,
                                                    const int32_t *__restrict__ c_pbeg, float4 *mac, float4 *mac_lo,
                                                    uint32_t *queue, unsigned long long *pool_ctr,
                                                    uint32_t *work_hist) {
  const int C = counts[0];
  if (blockIdx.x == 0) {  // the walk's group counters, list pool and cost histogram start empty
    if (threadIdx.x == 0) {
      queue[0] = 0;
      queue[1] = 0;
      pool_ctr[0] = 0;
    }
    for (int i = threadIdx.x; i < 2 * kCostBuckets; i += blockDim.x) work_hist[i] = 0;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    const Centre G = cell_centre<FOREST, DEEP>(c_level[c] & 31, c_pbeg[c], K, offs, S, frame, framef);
    mac[c] = make_float4(G.hi[0], G.hi[1], G.hi[2], 0.5f * G.l);
    if (DEEP) mac_lo[c] = make_float4(G.lo[0], G.lo[1], G.lo[2], 0.f);
  }
}

}  // namespace

template <bool FOREST, bool REFRESH, bool DEEP>
static void moments_impl(Ctx &c, cudaStream_t s) {
  const Keys K{c.key[0], c.skey_lo, c.levels};
  const int W = (int)((c.n + 31) / 32);  // the level scan's rows: W entries per level
  for (int k = c.levels; k >= 0; --k) {
    k_moments_level<FOREST, REFRESH, DEEP><<<c.num_sms * 4, kBlock, 0, s>>>(
        K, c.offs, c.n_sys, c.frame, c.framef, c.rowoff, W, k, c.c_level, c.c_pbeg, c.c_pend, c.c_first, c.c_nch,
        c.part_hi, c.part_lo, c.c_mom);
    c.launches++;
  }
}

template <bool REFRESH>
static void moments_launch(Ctx &c, cudaStream_t s) {
  const bool forest = c.n_sys > 1, deep = c.levels > kLevels;
  if (forest) deep ? moments_impl<true, REFRESH, true>(c, s) : moments_impl<true, REFRESH, false>(c, s);
  else deep ? moments_impl<false, REFRESH, true>(c, s) : moments_impl<false, REFRESH, false>(c, s);
}

template <bool FOREST, bool DEEP>
static void mac_box_impl(Ctx &c, cudaStream_t s) {
  const Keys K{c.key[0], c.skey_lo, c.levels};
  k_mac_box<FOREST, DEEP><<<c.num_sms * 8, kBlock, 0, s>>>(c.d_counts, K, c.offs, c.n_sys, c.frame, c.framef,
                                                           c.c_level, c.c_pbeg, c.c_mac, c.c_mac_lo, c.walk_queue,
                                                           c.pool_ctr, c.work_hist);
}

cudaError_t launch_moments(Ctx &c, cudaStream_t s) {
  moments_launch<false>(c, s);
  return cudaGetLastError();
}

cudaError_t launch_moments_refresh(Ctx &c, cudaStream_t s) {
  moments_launch<true>(c, s);
  return cudaGetLastError();
}

cudaError_t launch_mac(Ctx &c, float theta, cudaStream_t s) {
  float inv = (theta > 0.f) ? 1.0f / theta : INFINITY;
  if (c.p.mac == 1) {
    const bool forest = c.n_sys > 1, deep = c.levels > kLevels;
    if (forest) deep ? mac_box_impl<true, true>(c, s) : mac_box_impl<true, false>(c, s);
    else deep ? mac_box_impl<false, true>(c, s) : mac_box_impl<false, false>(c, s);
  } else {
    k_mac<<<c.num_sms * 8, kBlock, 0, s>>>(c.d_counts, c.c_mom, inv, c.c_mac, c.c_mac_lo, c.walk_queue, c.pool_ctr,
                                           c.work_hist);
  }
  c.launches++;
  return cudaGetLastError();
}

}  // namespace bh
