// k_direct.cu -- direct summation on the GPU (§4.2.1 measures the tree's
// accuracy against direct summation; §3.3: theta -> 0 turns the tree-code
// into a direct N-body code).
//
// Used as the product's own accuracy reference (the autotuner accepts a
// parameter set only if its error against this sum is no worse than the
// default's).  One thread per listed target; sources are staged 256 at a time
// in shared memory as two-float positions, and every pair difference is
// (s_hi - t_hi) + (s_lo - t_lo), so close pairs keep FP32 relative accuracy;
// tile sums are folded into (hi, lo) pairs by TwoSum.  The target itself is
// skipped by index.
#include <cuda_runtime.h>

#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ void fold2(float &hi, float &lo, float v) {
  float s = hi + v;
  float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

__global__ void __launch_bounds__(kBlock) k_direct(const double *__restrict__ pos, const double *__restrict__ mass,
                                                   int n, const int32_t *__restrict__ targets, int nt, float eps2,
                                                   float *acc, float *pot) {
  __shared__ float4 s_hi[kBlock];
  __shared__ float4 s_lo[kBlock];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = t < nt;
  const int me = ok ? targets[t] : -1;
  float th[3] = {0.f, 0.f, 0.f}, tl[3] = {0.f, 0.f, 0.f};
  if (ok)
    for (int a = 0; a < 3; ++a) split2(pos[3 * (size_t)me + a], th[a], tl[a]);
  float hx = 0, hy = 0, hz = 0, hp = 0, lx = 0, ly = 0, lz = 0, lp = 0;
  for (int base = 0; base < n; base += kBlock) {
    const int j = base + threadIdx.x;
    __syncthreads();
    if (j < n) {
      float h[3], l[3];
      for (int a = 0; a < 3; ++a) split2(pos[3 * (size_t)j + a], h[a], l[a]);
      s_hi[threadIdx.x] = make_float4(h[0], h[1], h[2], (float)mass[j]);
      s_lo[threadIdx.x] = make_float4(l[0], l[1], l[2], 0.f);
    }
    __syncthreads();
    const int cnt = min(kBlock, n - base);
    float ax = 0, ay = 0, az = 0, ap = 0;
    for (int q = 0; q < cnt; ++q) {
      const float4 sh = s_hi[q], sl = s_lo[q];
      float dx = (sh.x - th[0]) + (sl.x - tl[0]);
      float dy = (sh.y - th[1]) + (sl.y - tl[1]);
      float dz = (sh.z - th[2]) + (sl.z - tl[2]);
      float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
      float ri = (base + q == me || !(r2 > 0.f)) ? 0.f : rsqrtf(r2);
      float mr = sh.w * ri;
      float mr3 = mr * ri * ri;
      ap -= mr;
      ax = fmaf(mr3, dx, ax);
      ay = fmaf(mr3, dy, ay);
      az = fmaf(mr3, dz, az);
    }
    fold2(hx, lx, ax);
    fold2(hy, ly, ay);
    fold2(hz, lz, az);
    fold2(hp, lp, ap);
  }
  if (ok) {
    acc[3 * (size_t)t] = hx + lx;
    acc[3 * (size_t)t + 1] = hy + ly;
    acc[3 * (size_t)t + 2] = hz + lz;
    pot[t] = hp + lp;
  }
}

}  // namespace

cudaError_t launch_direct(const double *pos, const double *mass, int n, const int32_t *targets, int nt, float eps,
                          float *acc, float *pot, cudaStream_t s) {
  if (nt == 0) return cudaSuccess;
  k_direct<<<(nt + kBlock - 1) / kBlock, kBlock, 0, s>>>(pos, mass, n, targets, nt, eps * eps, acc, pot);
  return cudaGetLastError();
}

}  // namespace bh

extern "C" int bh_direct_forces(const double *pos_dev, const double *mass_dev, int64_t n, const int32_t *targets_dev,
                                int64_t nt, float eps, float *acc_dev, float *pot_dev, void *stream) {
  if (n < 0 || nt < 0 || n >= (1ll << 31) || nt >= (1ll << 31)) return BH_ERR_INVALID_ARG;
  if (nt > 0 && (!pos_dev || !mass_dev || !targets_dev || !acc_dev || !pot_dev)) return BH_ERR_INVALID_ARG;
  if (!(eps >= 0.f)) return BH_ERR_INVALID_ARG;
  cudaError_t e = bh::launch_direct(pos_dev, mass_dev, (int)n, targets_dev, (int)nt, eps, acc_dev, pot_dev,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}
