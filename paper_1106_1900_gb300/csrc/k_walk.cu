// k_walk.cu -- the breadth-first group walk and force evaluation (§2.2, §3.3).
//
// One warp walks one group (<= 64 bodies) at a time; warps take groups from
// a global counter (a persistent kernel), so the walk has no block-wide
// barrier at all.  Per group:
//
//  * every lane holds two target slots.  A group of more than 32 bodies maps
//    one body per slot; 17..32 bodies put each body in both slots of its lane
//    and split the sources between them; <= 16 bodies use four slots (two
//    lanes) per body and split the sources four ways -- the paper's
//    "several threads per particle" for small groups, with a final reduction.
//  * the current level of the walk is read 32 cells at a time from a
//    per-warp stack in global memory; each lane applies Eq. 1 to one cell
//    (d^2 > (l/theta + delta)^2, d = distance from the cell's centre of mass
//    to the group's bounding box).  Accepted cells are appended to the
//    cell list, opened nodes push their (contiguous) children on the next
//    level's stack, opened leaves append their (contiguous) bodies to the
//    particle list; the appends are warp ballots and warp prefix sums.
//  * whenever a list holds 32 entries they are staged in shared memory and
//    every lane sums the 32 interactions on its slots; the remainders are
//    flushed when the walk ends.
//
// Precision (variant 0): all coordinates are taken relative to the group
// centre c (a float: the first body's position), sources as
// (x_hi - c) + x_lo from their two-float form, so close pairs keep their
// relative accuracy; each 32-entry tile is summed in FP32 and tiles are
// added into a (hi, lo) pair by TwoSum.  Variant 1 is the naive form:
// absolute FP32 coordinates and plain sums.  A body is never paired with
// itself: particle tiles that hold bodies of the walking group (a ballot tells)
// run a loop that skips equal indices; all other tiles run the plain loop.
// With eps = 0 zero distances are skipped as well.
#include <cuda_runtime.h>

#include "bh_internal.cuh"

namespace bh {
namespace {

struct WarpSmem {
  int clist[64];
  int plist[64];
  float4 sc[36][3];  // staged cells: (dx, dy, dz, M), (Qxx, Qyy, Qzz, Qxy), (Qxz, Qyz, 0, 0)
  float4 sp[36];     // staged bodies: (dx, dy, dz, m)
  int pidx[36];      // their sorted indices (read only for tiles holding the group's own bodies)
};

struct WalkArgs {
  const float4 *__restrict__ part_hi;
  const float4 *__restrict__ part_lo;
  const float4 *__restrict__ mac;
  const int2 *__restrict__ link;
  const float4 *__restrict__ mom;
  const int32_t *__restrict__ g_beg;
  const int32_t *__restrict__ g_sys;
  const int32_t *__restrict__ sys_root;
  const int32_t *__restrict__ counts;
  int32_t *stack;
  int cap;
  int n;
  float eps2;
  uint32_t *queue;
  float4 *acc_sorted;
  float *acc_out;
  float *pot_out;
  const uint32_t *__restrict__ perm;
  int32_t *g_npc;
  int32_t *g_npp;
  unsigned long long *g_csum;
  unsigned long long *g_psum;
  unsigned long long *totals;
  int32_t *status;
};

constexpr float kFar = 1e18f;

struct Acc {
  float x, y, z, p;
};

__device__ __forceinline__ void two_sum_into(float &hi, float &lo, float v) {
  float s = hi + v;
  float bp = s - hi;
  float e = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += e;
}

template <int VAR>
__device__ __forceinline__ void fold_tile(Acc &hi, Acc &lo, const Acc &t) {
  if (VAR == 0) {
    two_sum_into(hi.x, lo.x, t.x);
    two_sum_into(hi.y, lo.y, t.y);
    two_sum_into(hi.z, lo.z, t.z);
    two_sum_into(hi.p, lo.p, t.p);
  } else {
    hi.x += t.x;
    hi.y += t.y;
    hi.z += t.z;
    hi.p += t.p;
  }
}

// Softened particle-particle interaction of source s = (dx, dy, dz, m) on a
// target at (tx, ty, tz): 20 flops by the convention FMA = 2, rsqrt = 1.
// SELF: the tile holds bodies of the walking group, so the pair of a body
// with itself (same index) is skipped; GUARD: eps = 0, zero distances skipped.
template <bool GUARD, bool SELF = false>
__device__ __forceinline__ void pp(Acc &a, float tx, float ty, float tz, const float4 s, float eps2,
                                   int me = 0, int other = 1) {
  float dx = s.x - tx, dy = s.y - ty, dz = s.z - tz;
  float r2 = fmaf(dx, dx, eps2);
  r2 = fmaf(dy, dy, r2);
  r2 = fmaf(dz, dz, r2);
  float ri = rsqrtf(r2);
  if (GUARD) ri = (r2 > 0.f) ? ri : 0.f;
  if (SELF) ri = (me == other) ? 0.f : ri;
  float mr = s.w * ri;
  float mr3 = mr * ri * ri;
  a.p -= mr;
  a.x = fmaf(mr3, dx, a.x);
  a.y = fmaf(mr3, dy, a.y);
  a.z = fmaf(mr3, dz, a.z);
}

// Softened particle-cell interaction, monopole + quadrupole, with d = com -
// target: a = M d/s^3 - Q d/s^5 + (5/2)(d.Q.d) d/s^7, phi = -M/s - (d.Q.d)/(2 s^5).
__device__ __forceinline__ void pc(Acc &a, float tx, float ty, float tz, const float4 c0, const float4 q0,
                                   const float4 q1, float eps2) {
  float dx = c0.x - tx, dy = c0.y - ty, dz = c0.z - tz;
  float r2 = fmaf(dx, dx, eps2);
  r2 = fmaf(dy, dy, r2);
  r2 = fmaf(dz, dz, r2);
  float ri = rsqrtf(r2);
  float ri2 = ri * ri;
  float mr = c0.w * ri;
  float mr3 = mr * ri2;
  float qx = fmaf(q1.x, dz, fmaf(q0.w, dy, q0.x * dx));
  float qy = fmaf(q1.y, dz, fmaf(q0.y, dy, q0.w * dx));
  float qz = fmaf(q0.z, dz, fmaf(q1.y, dy, q1.x * dx));
  float dqd = fmaf(qz, dz, fmaf(qy, dy, qx * dx));
  float ri5 = ri2 * ri2 * ri;
  float qr5 = dqd * ri5;
  a.p = fmaf(-0.5f, qr5, a.p - mr);
  float coef = fmaf(2.5f * qr5, ri2, mr3);
  a.x = fmaf(-ri5, qx, fmaf(coef, dx, a.x));
  a.y = fmaf(-ri5, qy, fmaf(coef, dy, a.y));
  a.z = fmaf(-ri5, qz, fmaf(coef, dz, a.z));
}

template <int VAR, bool GUARD, int MODE>
__global__ void k_walk(WalkArgs A) {
  extern __shared__ WarpSmem s_warp[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  WarpSmem &S = s_warp[wib];
  const size_t gw = (size_t)blockIdx.x * (blockDim.x >> 5) + wib;
  int *cur = A.stack + gw * 2 * (size_t)A.cap;
  int *nxt = cur + A.cap;
  const unsigned lt = lanemask_lt();
  const float eps2 = A.eps2;
  if (lane < 4) {
    S.sc[32 + lane][0] = make_float4(kFar, kFar, kFar, 0.f);
    S.sc[32 + lane][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    S.sc[32 + lane][2] = make_float4(0.f, 0.f, 0.f, 0.f);
    S.sp[32 + lane] = make_float4(kFar, kFar, kFar, 0.f);
    S.pidx[32 + lane] = -1;
  }
  __syncwarp();
  const int G = A.counts[1];

  while (true) {
    int g = 0;
    if (lane == 0) g = (int)atomicAdd(A.queue, 1u);
    g = __shfl_sync(kFull, g, 0);
    if (g >= G) break;
    const int gb = A.g_beg[g];
    const int n = A.g_beg[g + 1] - gb;
    const int root = A.sys_root[A.g_sys[g]];
    const int tpp = (n <= 16) ? 4 : ((n <= 32) ? 2 : 1);
    int p0, p1, ph0;
    if (tpp == 1) {
      p0 = lane;
      p1 = lane + 32;
      ph0 = 0;
    } else if (tpp == 2) {
      p0 = p1 = lane;
      ph0 = 0;
    } else {
      p0 = p1 = lane & 15;
      ph0 = lane >> 4;
    }
    const bool v0 = p0 < n, v1 = p1 < n;
    // group centre and targets (same arithmetic as the staged sources)
    float cx = 0.f, cy = 0.f, cz = 0.f;
    if (VAR == 0) {
      float4 c = A.part_hi[gb];
      cx = c.x;
      cy = c.y;
      cz = c.z;
    }
    float t0x, t0y, t0z, t1x, t1y, t1z;
    {
      float4 h = A.part_hi[gb + min(p0, n - 1)], l = A.part_lo[gb + min(p0, n - 1)];
      if (VAR == 0) {
        t0x = (h.x - cx) + l.x;
        t0y = (h.y - cy) + l.y;
        t0z = (h.z - cz) + l.z;
      } else {
        t0x = h.x;
        t0y = h.y;
        t0z = h.z;
      }
      h = A.part_hi[gb + min(p1, n - 1)];
      l = A.part_lo[gb + min(p1, n - 1)];
      if (VAR == 0) {
        t1x = (h.x - cx) + l.x;
        t1y = (h.y - cy) + l.y;
        t1z = (h.z - cz) + l.z;
      } else {
        t1x = h.x;
        t1y = h.y;
        t1z = h.z;
      }
    }
    // tight bounding box of the group's bodies
    float bminx = fminf(v0 ? t0x : INFINITY, v1 ? t1x : INFINITY);
    float bminy = fminf(v0 ? t0y : INFINITY, v1 ? t1y : INFINITY);
    float bminz = fminf(v0 ? t0z : INFINITY, v1 ? t1z : INFINITY);
    float bmaxx = fmaxf(v0 ? t0x : -INFINITY, v1 ? t1x : -INFINITY);
    float bmaxy = fmaxf(v0 ? t0y : -INFINITY, v1 ? t1y : -INFINITY);
    float bmaxz = fmaxf(v0 ? t0z : -INFINITY, v1 ? t1z : -INFINITY);
    for (int o = 16; o > 0; o >>= 1) {
      bminx = fminf(bminx, __shfl_xor_sync(kFull, bminx, o));
      bminy = fminf(bminy, __shfl_xor_sync(kFull, bminy, o));
      bminz = fminf(bminz, __shfl_xor_sync(kFull, bminz, o));
      bmaxx = fmaxf(bmaxx, __shfl_xor_sync(kFull, bmaxx, o));
      bmaxy = fmaxf(bmaxy, __shfl_xor_sync(kFull, bmaxy, o));
      bmaxz = fmaxf(bmaxz, __shfl_xor_sync(kFull, bmaxz, o));
    }
    Acc h0 = {0, 0, 0, 0}, l0 = {0, 0, 0, 0}, h1 = {0, 0, 0, 0}, l1 = {0, 0, 0, 0};
    int cn = 0, pn = 0, ncell = 0, npart = 0;
    unsigned long long csum = 0, psum = 0;

    // ---- evaluate the first `cnt` entries of the cell list
    auto eval_cells = [&](int cnt) {
      if (lane < cnt) {
        int cc = S.clist[lane];
        float4 a = A.mom[4 * (size_t)cc], b = A.mom[4 * (size_t)cc + 1];
        float4 q0 = A.mom[4 * (size_t)cc + 2], q1 = A.mom[4 * (size_t)cc + 3];
        float dx, dy, dz;
        if (VAR == 0) {
          dx = (a.x - cx) + b.x;
          dy = (a.y - cy) + b.y;
          dz = (a.z - cz) + b.z;
        } else {
          dx = a.x;
          dy = a.y;
          dz = a.z;
        }
        S.sc[lane][0] = make_float4(dx, dy, dz, a.w);
        S.sc[lane][1] = q0;
        S.sc[lane][2] = make_float4(q1.x, q1.y, 0.f, 0.f);
      } else {
        S.sc[lane][0] = make_float4(kFar, kFar, kFar, 0.f);
        S.sc[lane][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        S.sc[lane][2] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();
      Acc t0 = {0, 0, 0, 0}, t1 = {0, 0, 0, 0};
      if (tpp == 1) {
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
          const float4 c0 = S.sc[j][0], q0 = S.sc[j][1], q1 = S.sc[j][2];
          pc(t0, t0x, t0y, t0z, c0, q0, q1, eps2);
          pc(t1, t1x, t1y, t1z, c0, q0, q1, eps2);
        }
      } else if (tpp == 2) {
#pragma unroll 2
        for (int j = 0; j < cnt; j += 2) {
          pc(t0, t0x, t0y, t0z, S.sc[j][0], S.sc[j][1], S.sc[j][2], eps2);
          pc(t1, t1x, t1y, t1z, S.sc[j + 1][0], S.sc[j + 1][1], S.sc[j + 1][2], eps2);
        }
      } else {
#pragma unroll 2
        for (int j = 0; j < cnt; j += 4) {
          const int s0 = j + ph0, s1 = j + ph0 + 2;
          pc(t0, t0x, t0y, t0z, S.sc[s0][0], S.sc[s0][1], S.sc[s0][2], eps2);
          pc(t1, t1x, t1y, t1z, S.sc[s1][0], S.sc[s1][1], S.sc[s1][2], eps2);
        }
      }
      fold_tile<VAR>(h0, l0, t0);
      fold_tile<VAR>(h1, l1, t1);
      __syncwarp();
    };

    // ---- evaluate the first `cnt` entries of the particle list
    auto eval_bodies = [&](int cnt) {
      bool member = false;
      if (lane < cnt) {
        int b = S.plist[lane];
        member = (unsigned)(b - gb) < (unsigned)n;
        float4 h = A.part_hi[b], l = A.part_lo[b];
        if (VAR == 0)
          S.sp[lane] = make_float4((h.x - cx) + l.x, (h.y - cy) + l.y, (h.z - cz) + l.z, h.w);
        else
          S.sp[lane] = h;
        S.pidx[lane] = b;
      } else {
        S.sp[lane] = make_float4(kFar, kFar, kFar, 0.f);
        S.pidx[lane] = -1;
      }
      const bool self_tile = __any_sync(kFull, member);
      __syncwarp();
      Acc t0 = {0, 0, 0, 0}, t1 = {0, 0, 0, 0};
      if (self_tile) {
        // a tile with the group's own bodies: skip each body's pair with itself by index
        const int me0 = gb + p0, me1 = gb + p1;
        const int st = (tpp == 1) ? 1 : tpp;
        const int o0 = (tpp == 1) ? 0 : ph0, o1 = (tpp == 1) ? 0 : ((tpp == 2) ? 1 : ph0 + 2);
        for (int j = 0; j < cnt; j += st) {
          pp<GUARD, true>(t0, t0x, t0y, t0z, S.sp[j + o0], eps2, me0, S.pidx[j + o0]);
          pp<GUARD, true>(t1, t1x, t1y, t1z, S.sp[j + o1], eps2, me1, S.pidx[j + o1]);
        }
      } else if (tpp == 1) {
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
          const float4 s = S.sp[j];
          pp<GUARD>(t0, t0x, t0y, t0z, s, eps2);
          pp<GUARD>(t1, t1x, t1y, t1z, s, eps2);
        }
      } else if (tpp == 2) {
#pragma unroll 4
        for (int j = 0; j < cnt; j += 2) {
          pp<GUARD>(t0, t0x, t0y, t0z, S.sp[j], eps2);
          pp<GUARD>(t1, t1x, t1y, t1z, S.sp[j + 1], eps2);
        }
      } else {
#pragma unroll 4
        for (int j = 0; j < cnt; j += 4) {
          pp<GUARD>(t0, t0x, t0y, t0z, S.sp[j + ph0], eps2);
          pp<GUARD>(t1, t1x, t1y, t1z, S.sp[j + ph0 + 2], eps2);
        }
      }
      fold_tile<VAR>(h0, l0, t0);
      fold_tile<VAR>(h1, l1, t1);
      __syncwarp();
    };

    // ---- breadth-first walk (§2.2)
    if (lane == 0) cur[0] = root;
    __syncwarp();
    int ncur = 1;
    int *cstk = cur, *nstk = nxt;
    int depth = 0;
    while (ncur > 0) {
      if (++depth > kLevels + 1) {  // a tree has at most 21 levels: never loop on a corrupt one
        if (lane == 0) set_status(A.status, BH_ERR_STATE);
        break;
      }
      int nnext = 0;
      for (int base = 0; base < ncur; base += 32) {
        const bool have = base + lane < ncur;
        int ci = 0;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        int2 lk = make_int2(0, 0);
        if (have) {
          ci = cstk[base + lane];
          m = A.mac[ci];
          lk = A.link[ci];
        }
        float rx = m.x - cx, ry = m.y - cy, rz = m.z - cz;
        float ex = fmaxf(fmaxf(bminx - rx, rx - bmaxx), 0.f);
        float ey = fmaxf(fmaxf(bminy - ry, ry - bmaxy), 0.f);
        float ez = fmaxf(fmaxf(bminz - rz, rz - bmaxz), 0.f);
        float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const bool accept = have && d2 > m.w * m.w;
        const bool open = have && !accept;
        const bool leaf = lk.y < 0;
        // accepted cells -> cell list
        unsigned ab = __ballot_sync(kFull, accept);
        if (accept) {
          S.clist[cn + __popc(ab & lt)] = ci;
          csum += (unsigned long long)ci;
        }
        cn += __popc(ab);
        ncell += __popc(ab);
        __syncwarp();
        if (cn >= 32) {
          eval_cells(32);
          int tmp = (lane < cn - 32) ? S.clist[32 + lane] : 0;
          __syncwarp();
          if (lane < cn - 32) S.clist[lane] = tmp;
          cn -= 32;
          __syncwarp();
        }
        // opened nodes -> children on the next level
        int nch = (open && !leaf) ? min(max(lk.y, 0), 8) : 0;
        int inc = nch;
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(kFull, inc, o);
          if (lane >= o) inc += y;
        }
        const int tot = __shfl_sync(kFull, inc, 31);
        if (nnext + tot <= A.cap) {
          for (int j = 0; j < nch; ++j) nstk[nnext + inc - nch + j] = lk.x + j;
          nnext += tot;
        } else if (tot > 0) {
          if (lane == 0) set_status(A.status, BH_ERR_CAPACITY);
        }
        // opened leaves -> bodies on the particle list
        int np = (open && leaf) ? (lk.y & 0x7fffffff) : 0;
        int pin = np;
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(kFull, pin, o);
          if (lane >= o) pin += y;
        }
        int ptot = __shfl_sync(kFull, pin, 31);
        if (ptot < 0 || ptot > A.n) {  // more bodies than exist: a corrupt link word
          if (lane == 0) set_status(A.status, BH_ERR_STATE);
          ptot = 0;
        }
        npart += ptot;
        const int pex = pin - np;
        for (int cb = 0; cb < ptot; cb += 32) {
          const int si = cb + lane;
          int k = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            int v = __shfl_sync(kFull, pin, k + step - 1);
            if (v <= si) k += step;
          }
          const int of = __shfl_sync(kFull, lk.x, k);
          const int oe = __shfl_sync(kFull, pex, k);
          if (si < ptot) {
            const int body = of + (si - oe);
            S.plist[pn + lane] = body;
            psum += (unsigned long long)body;
          }
          pn += min(32, ptot - cb);
          __syncwarp();
          if (pn >= 32) {
            eval_bodies(32);
            int tmp = (lane < pn - 32) ? S.plist[32 + lane] : 0;
            __syncwarp();
            if (lane < pn - 32) S.plist[lane] = tmp;
            pn -= 32;
            __syncwarp();
          }
        }
      }
      __syncwarp();
      int *t = cstk;
      cstk = nstk;
      nstk = t;
      ncur = nnext;
    }
    if (cn > 0) eval_cells(cn);
    if (pn > 0) eval_bodies(pn);

    // ---- combine the slots of each body and write
    float ox, oy, oz, op;
    if (tpp == 1) {
      // slot 0: body p0, slot 1: body p1
      if (v0 || v1) {
        Acc r[2] = {{h0.x + l0.x, h0.y + l0.y, h0.z + l0.z, h0.p + l0.p},
                    {h1.x + l1.x, h1.y + l1.y, h1.z + l1.z, h1.p + l1.p}};
        const int pb[2] = {p0, p1};
        const bool vv[2] = {v0, v1};
        for (int s = 0; s < 2; ++s) {
          if (!vv[s]) continue;
          const int b = gb + pb[s];
          if (MODE == kOutSorted) {
            A.acc_sorted[b] = make_float4(r[s].x, r[s].y, r[s].z, r[s].p);
          } else {
            const size_t j = A.perm[b];
            A.acc_out[3 * j] = r[s].x;
            A.acc_out[3 * j + 1] = r[s].y;
            A.acc_out[3 * j + 2] = r[s].z;
            A.pot_out[j] = r[s].p;
          }
        }
      }
    } else {
      // both slots hold the same body: combine them (and, with four slots, the partner lane)
      two_sum_into(h0.x, l0.x, h1.x);
      two_sum_into(h0.y, l0.y, h1.y);
      two_sum_into(h0.z, l0.z, h1.z);
      two_sum_into(h0.p, l0.p, h1.p);
      l0.x += l1.x;
      l0.y += l1.y;
      l0.z += l1.z;
      l0.p += l1.p;
      if (tpp == 4) {
        float ux = __shfl_xor_sync(kFull, h0.x, 16), uy = __shfl_xor_sync(kFull, h0.y, 16);
        float uz = __shfl_xor_sync(kFull, h0.z, 16), up = __shfl_xor_sync(kFull, h0.p, 16);
        float wx = __shfl_xor_sync(kFull, l0.x, 16), wy = __shfl_xor_sync(kFull, l0.y, 16);
        float wz = __shfl_xor_sync(kFull, l0.z, 16), wp = __shfl_xor_sync(kFull, l0.p, 16);
        two_sum_into(h0.x, l0.x, ux);
        two_sum_into(h0.y, l0.y, uy);
        two_sum_into(h0.z, l0.z, uz);
        two_sum_into(h0.p, l0.p, up);
        l0.x += wx;
        l0.y += wy;
        l0.z += wz;
        l0.p += wp;
      }
      ox = h0.x + l0.x;
      oy = h0.y + l0.y;
      oz = h0.z + l0.z;
      op = h0.p + l0.p;
      const bool writer = v0 && (tpp == 2 || lane < 16);
      if (writer) {
        const int b = gb + p0;
        if (MODE == kOutSorted) {
          A.acc_sorted[b] = make_float4(ox, oy, oz, op);
        } else {
          const size_t j = A.perm[b];
          A.acc_out[3 * j] = ox;
          A.acc_out[3 * j + 1] = oy;
          A.acc_out[3 * j + 2] = oz;
          A.pot_out[j] = op;
        }
      }
    }
    // ---- group statistics
    for (int o = 16; o > 0; o >>= 1) {
      csum += __shfl_xor_sync(kFull, csum, o);
      psum += __shfl_xor_sync(kFull, psum, o);
    }
    if (lane == 0) {
      A.g_npc[g] = ncell;
      A.g_npp[g] = npart;
      A.g_csum[g] = csum;
      A.g_psum[g] = psum;
      // every body of the group is on its own particle list once (its own
      // leaves are always opened for theta < 1.15): that self pair is not counted
      const unsigned long long self = (npart >= n) ? (unsigned long long)n : 0ull;
      atomicAdd(&A.totals[0], (unsigned long long)n * (unsigned long long)npart - self);
      atomicAdd(&A.totals[1], (unsigned long long)n * (unsigned long long)ncell);
    }
  }
}

template <int VAR, bool GUARD, int MODE>
cudaError_t launch_one(Ctx &c, const WalkArgs &a, cudaStream_t s) {
  k_walk<VAR, GUARD, MODE><<<c.walk_grid, c.p.walk_warps * 32, c.walk_smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int walk_smem_bytes(int warps) { return warps * (int)sizeof(WarpSmem); }

cudaError_t walk_init_attrs(int smem) {
  cudaError_t e = cudaSuccess;
#define BH_WALK_ATTR(V, G, M) \
  if (!e) e = cudaFuncSetAttribute(k_walk<V, G, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  BH_WALK_ATTR(0, false, kOutCaller)
  BH_WALK_ATTR(0, true, kOutCaller)
  BH_WALK_ATTR(0, false, kOutSorted)
  BH_WALK_ATTR(0, true, kOutSorted)
  BH_WALK_ATTR(1, false, kOutCaller)
  BH_WALK_ATTR(1, true, kOutCaller)
  BH_WALK_ATTR(1, false, kOutSorted)
  BH_WALK_ATTR(1, true, kOutSorted)
#undef BH_WALK_ATTR
  return e;
}

int walk_max_blocks_per_sm(int warps, int smem) {
  int nb = 0;
  cudaFuncSetAttribute(k_walk<0, false, kOutCaller>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk<0, false, kOutCaller>, warps * 32, smem) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_walk(Ctx &c, float eps, OutMode mode, float *acc, float *pot, cudaStream_t s) {
  WalkArgs a;
  a.part_hi = c.part_hi;
  a.part_lo = c.part_lo;
  a.mac = c.c_mac;
  a.link = c.c_link;
  a.mom = c.c_mom;
  a.g_beg = c.g_beg;
  a.g_sys = c.g_sys;
  a.sys_root = c.sys_root;
  a.counts = c.d_counts;
  a.stack = c.walk_stack;
  a.cap = c.p.stack_capacity;
  a.n = (int)c.n;
  a.eps2 = eps * eps;
  a.queue = c.walk_queue;
  a.acc_sorted = c.acc_sorted;
  a.acc_out = acc;
  a.pot_out = pot;
  a.perm = c.idx[0];
  a.g_npc = c.g_npc;
  a.g_npp = c.g_npp;
  a.g_csum = c.g_csum;
  a.g_psum = c.g_psum;
  a.totals = c.d_totals;
  a.status = c.d_status;
  const bool guard = !(a.eps2 > 0.f);
  const int var = c.p.walk_variant;
  cudaError_t e;
#define BH_WALK_CASE(V, G, M) \
  if (var == V && guard == G && mode == M) e = launch_one<V, G, M>(c, a, s); else
  BH_WALK_CASE(0, false, kOutCaller)
  BH_WALK_CASE(0, true, kOutCaller)
  BH_WALK_CASE(0, false, kOutSorted)
  BH_WALK_CASE(0, true, kOutSorted)
  BH_WALK_CASE(1, false, kOutCaller)
  BH_WALK_CASE(1, true, kOutCaller)
  BH_WALK_CASE(1, false, kOutSorted)
  BH_WALK_CASE(1, true, kOutSorted)
  e = cudaErrorInvalidValue;
#undef BH_WALK_CASE
  c.launches++;
  return e;
}

}  // namespace bh
