// k_block.cu -- block time-steps (the paper's motivation for building the
// whole tree code on the GPU, §1, §2.2, §4): every body steps with
// dt_max 2^-k (its level k), times are integer ticks of dt_max 2^-k_max, a
// block step advances to the earliest time a body is due, walks only the
// groups that hold a due ("active") body and corrects only the active bodies;
// between rebuilds the tree is kept and its moments are refreshed.
//
//   k_block_levels   first levels (and time 0) after the forces at t = 0
//   k_block_next     block time T = min over bodies of (t_i + 2^(k_max - k_i))
//   k_block_predict  every body predicted to T (the leapfrog predictor of
//                    k_predict, operation for operation), active bodies counted
//   k_move_block     a rebuild's permutation of the state, ticks and levels;
//                    the tree's bodies from the predicted positions
//   k_block_parts    a refresh: the tree's bodies from the predicted positions
//   k_group_active   groups holding an active body
//   k_block_correct  active bodies: the leapfrog corrector of k_correct, then
//                    the level rule (deeper at once, shallower by one level
//                    when T is a multiple of the doubled step)
#include <cuda_runtime.h>

#include <cmath>

#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kBlock = 256;

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ long long step_ticks(int kmax, int k) { return 1ll << (kmax - k); }

// The level a body with acceleration a wants: the smallest k >= 0 with
// dt_max 2^-k <= eta sqrt(eps / |a|), i.e. 2^k >= r = c |a|^(1/2) with
// c = dt_max / (eta sqrt(eps)) (from the host, FP64 rounded to float); in
// FP32, as the accelerations are, with k read from r's exponent bits (r is
// then a normal float above 1); clamped to kmax.  NaN gives 0.
__device__ __forceinline__ int wanted_level(float4 a, float c, int kmax) {
  const float s = fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z));
  const float r = c * sqrtf(sqrtf(s));
  if (!(r > 1.f)) return 0;
  const unsigned b = __float_as_uint(r);
  const int e = (int)((b >> 23) & 0xffu) - 127;  // r = 1.f 2^e
  const int k = (b & 0x7fffffu) ? e + 1 : e;     // a power of two needs no more
  return min(k, kmax);
}

__global__ void __launch_bounds__(kBlock) k_block_levels(int n, const float4 *__restrict__ a, int64_t *t, int32_t *k,
                                                         float c_level, int kmax, unsigned long long *blk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) blk[0] = 0;
  unsigned lv = 0;
  if (i < n) {
    t[i] = 0;
    lv = (unsigned)wanted_level(a[i], c_level, kmax);
    k[i] = (int32_t)lv;
  }
  // deepest level: one atomic per warp (one per body serialises on one address)
  lv = __reduce_max_sync(kFull, lv);
  if ((threadIdx.x & 31) == 0) atomicMax(&blk[2], (unsigned long long)lv);
}

// blk[0] = min over bodies of the next due time (blk[0] preset to all ones)
__global__ void __launch_bounds__(kBlock) k_block_next(int n, const int64_t *__restrict__ t,
                                                       const int32_t *__restrict__ k, int kmax,
                                                       unsigned long long *blk) {
  __shared__ unsigned long long s_min[kBlock / 32];
  unsigned long long m = ~0ull;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = min(m, (unsigned long long)(t[i] + step_ticks(kmax, k[i])));
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kBlock / 32; ++w) m = min(m, s_min[w]);
    atomicMin(&blk[0], m);
  }
}

__global__ void __launch_bounds__(kBlock) k_block_predict(int n, const double *__restrict__ x,
                                                          const double *__restrict__ v, const float4 *__restrict__ a,
                                                          const int64_t *__restrict__ t,
                                                          const int32_t *__restrict__ k, int kmax, double tick,
                                                          unsigned long long *blk, double *pred) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long long T = (long long)blk[0];
  bool act = false;
  if (i < n) {
    act = t[i] + step_ticks(kmax, k[i]) == T;
    const double dt = (double)(T - t[i]) * tick;
    const float4 ai = a[i];
    const double ac[3] = {(double)ai.x, (double)ai.y, (double)ai.z};
    const double hdt2 = 0.5 * dt * dt;
    for (int d = 0; d < 3; ++d) {
      const size_t q = 3 * (size_t)i + d;
      pred[q] = x[q] + v[q] * dt + ac[d] * hdt2;
    }
  }
  const unsigned b = __ballot_sync(kFull, act);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&blk[1], (unsigned long long)__popc(b));
}

__global__ void __launch_bounds__(kBlock) k_move_block(const uint32_t *__restrict__ perm, int n,
                                                       const double *__restrict__ x0, const double *__restrict__ v0,
                                                       const double *__restrict__ m0, const float4 *__restrict__ a0,
                                                       const int32_t *__restrict__ id0,
                                                       const int64_t *__restrict__ t0, const int32_t *__restrict__ k0,
                                                       const double *__restrict__ pred, double *x1, double *v1,
                                                       double *m1, float4 *a1, int32_t *id1, int64_t *t1, int32_t *k1,
                                                       double *pred_s, float4 *part_hi, float4 *part_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t j = perm[i];
  float h[3], l[3];
  for (int a = 0; a < 3; ++a) {
    x1[3 * (size_t)i + a] = x0[3 * j + a];
    v1[3 * (size_t)i + a] = v0[3 * j + a];
    const double p = pred[3 * j + a];
    pred_s[3 * (size_t)i + a] = p;
    split2(p, h[a], l[a]);
  }
  const double m = m0[j];
  m1[i] = m;
  a1[i] = a0[j];
  id1[i] = id0[j];
  t1[i] = t0[j];
  k1[i] = k0[j];
  part_hi[i] = make_float4(h[0], h[1], h[2], (float)m);
  part_lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

__global__ void __launch_bounds__(kBlock) k_block_parts(int n, const double *__restrict__ pred,
                                                        const double *__restrict__ m, float4 *part_hi,
                                                        float4 *part_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float h[3], l[3];
  for (int a = 0; a < 3; ++a) split2(pred[3 * (size_t)i + a], h[a], l[a]);
  part_hi[i] = make_float4(h[0], h[1], h[2], (float)m[i]);
  part_lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

__global__ void __launch_bounds__(kBlock) k_group_active(const int32_t *__restrict__ counts,
                                                         const int32_t *__restrict__ g_beg,
                                                         const int64_t *__restrict__ t,
                                                         const int32_t *__restrict__ k, int kmax,
                                                         const unsigned long long *__restrict__ blk,
                                                         uint8_t *g_active) {
  const int G = counts[1];
  const long long T = (long long)blk[0];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    uint8_t on = 0;
    for (int i = g_beg[g]; i < g_beg[g + 1] && !on; ++i) on = (t[i] + step_ticks(kmax, k[i]) == T);
    g_active[g] = on;
  }
}

// One due body: the leapfrog corrector of k_correct, then the level rule;
// returns the new level.
__device__ __forceinline__ unsigned correct_body(int i, long long s, long long T, double *x, double *v,
                                                 float4 *a_old, int64_t *t, int32_t *k,
                                                 const float4 *__restrict__ a_new, const double *__restrict__ pred,
                                                 int kmax, double tick, float c_level) {
  const double dt = (double)s * tick;
  const float4 o = a_old[i], w = a_new[i];
  const double h = 0.5 * dt;
  const double ao[3] = {(double)o.x, (double)o.y, (double)o.z};
  const double an[3] = {(double)w.x, (double)w.y, (double)w.z};
  for (int d = 0; d < 3; ++d) {
    const size_t q = 3 * (size_t)i + d;
    const double vp = v[q] + ao[d] * dt;
    v[q] = vp + (an[d] - ao[d]) * h;
    x[q] = pred[q];
  }
  a_old[i] = w;
  t[i] = T;
  // level rule: deeper at once; one level shallower when T is a multiple of the doubled step
  const int want = wanted_level(w, c_level, kmax);
  int kn = k[i];
  if (want > kn) kn = want;
  else if (want < kn && kn > 0 && T % (2 * s) == 0) kn = kn - 1;
  k[i] = kn;
  return (unsigned)kn;
}

__global__ void __launch_bounds__(kBlock) k_block_correct(int n, double *x, double *v, float4 *a_old,
                                                          int64_t *t, int32_t *k, const float4 *__restrict__ a_new,
                                                          const double *__restrict__ pred, int kmax, double tick,
                                                          float c_level, unsigned long long *blk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long long T = (long long)blk[0];
  const long long s = (i < n) ? step_ticks(kmax, k[i]) : 0;
  const bool act = i < n && t[i] + s == T;
  const unsigned kn = act ? correct_body(i, s, T, x, v, a_old, t, k, a_new, pred, kmax, tick, c_level) : 0u;
  // deepest level: one atomic per warp (one per body serialises on one address)
  const unsigned km = __reduce_max_sync(kFull, kn);
  if ((threadIdx.x & 31) == 0 && __any_sync(kFull, act)) atomicMax(&blk[2], (unsigned long long)km);
}

// levels and ticks in the caller's order
__global__ void __launch_bounds__(kBlock) k_block_get(int n, const int32_t *__restrict__ id,
                                                      const int32_t *__restrict__ k, const int64_t *__restrict__ t,
                                                      int32_t *level, int64_t *tick) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = id[i];
  if (level) level[j] = k[i];
  if (tick) tick[j] = t[i];
}

}  // namespace

// c = dt_max / (eta sqrt(eps)) of the level rule
static float level_factor(const Ctx &c, double eps) { return (float)(c.blk_dt_max / (c.blk_eta * std::sqrt(eps))); }

cudaError_t launch_block_get(Ctx &c, int32_t *level, int64_t *tick, cudaStream_t s) {
  const int a = c.state_cur;
  k_block_get<<<cdiv(c.n, kBlock), kBlock, 0, s>>>((int)c.n, c.st_id[a], c.st_k[a], c.st_t[a], level, tick);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_block_levels(Ctx &c, double eps, cudaStream_t s) {
  const int a = c.state_cur;
  cudaError_t e = cudaMemsetAsync(c.d_block, 0, 4 * sizeof(unsigned long long), s);
  if (e) return e;
  k_block_levels<<<cdiv(c.n, kBlock), kBlock, 0, s>>>((int)c.n, c.st_a[a], c.st_t[a], c.st_k[a],
                                                      level_factor(c, eps), c.blk_kmax, c.d_block);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_block_predict(Ctx &c, cudaStream_t s) {
  const int a = c.state_cur;
  cudaError_t e = cudaMemsetAsync(c.d_block, 0xff, sizeof(unsigned long long), s);
  if (!e) e = cudaMemsetAsync(c.d_block + 1, 0, 2 * sizeof(unsigned long long), s);
  if (e) return e;
  k_block_next<<<c.num_sms * 4, kBlock, 0, s>>>((int)c.n, c.st_t[a], c.st_k[a], c.blk_kmax, c.d_block);
  k_block_predict<<<cdiv(c.n, kBlock), kBlock, 0, s>>>((int)c.n, c.st_x[a], c.st_v[a], c.st_a[a], c.st_t[a],
                                                       c.st_k[a], c.blk_kmax, c.blk_tick, c.d_block, c.pred_x);
  c.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_move_block(Ctx &c, cudaStream_t s) {
  const int a = c.state_cur, b = a ^ 1;
  k_move_block<<<cdiv(c.n, kBlock), kBlock, 0, s>>>(c.idx[0], (int)c.n, c.st_x[a], c.st_v[a], c.st_m[a], c.st_a[a],
                                                    c.st_id[a], c.st_t[a], c.st_k[a], c.pred_x, c.st_x[b], c.st_v[b],
                                                    c.st_m[b], c.st_a[b], c.st_id[b], c.st_t[b], c.st_k[b],
                                                    c.pred_s, c.part_hi, c.part_lo);
  c.state_cur = b;
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_block_parts(Ctx &c, cudaStream_t s) {
  k_block_parts<<<cdiv(c.n, kBlock), kBlock, 0, s>>>((int)c.n, c.pred_x, c.st_m[c.state_cur], c.part_hi,
                                                     c.part_lo);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_group_active(Ctx &c, cudaStream_t s) {
  const int a = c.state_cur;
  k_group_active<<<c.num_sms * 4, kBlock, 0, s>>>(c.d_counts, c.g_beg, c.st_t[a], c.st_k[a], c.blk_kmax, c.d_block,
                                                  c.g_active);
  c.launches++;
  return cudaGetLastError();
}

cudaError_t launch_block_correct(Ctx &c, double eps, bool rebuilt, cudaStream_t s) {
  const int a = c.state_cur;
  k_block_correct<<<cdiv(c.n, kBlock), kBlock, 0, s>>>((int)c.n, c.st_x[a], c.st_v[a], c.st_a[a], c.st_t[a],
                                                       c.st_k[a], c.acc_sorted, rebuilt ? c.pred_s : c.pred_x,
                                                       c.blk_kmax, c.blk_tick, level_factor(c, eps), c.d_block);
  c.launches++;
  return cudaGetLastError();
}

}  // namespace bh
