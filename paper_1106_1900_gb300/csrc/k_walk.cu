// k_walk.cu -- the breadth-first group walk and force evaluation (§2.2, §3.3).
//
// One warp walks one group (<= 64 bodies) at a time; warps take groups from
// a global counter (a persistent kernel), so the walk has no block-wide
// barrier at all.  Per group:
//
//  * every lane holds two target slots, 64 per warp.  A group of n bodies
//    gets k = floor(64/n) slots per body (one for n > 32): slot s holds body
//    s mod n and takes every k-th source starting at s div n, and the slots of
//    a body are summed when the group ends -- the paper's "several threads
//    per particle" for small groups, generalised so that few slots idle.
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
// Precision (variant 0): coordinates are offsets from the group centre c (a
// float: the first body's position), each kept as two floats -- the rounded
// offset and its exact residual -- built from the two-float body positions.
// Particle-particle terms difference both parts, so a close pair stays
// accurate however far from c it lies; particle-cell terms use the rounded
// part (accepted cells lie at least l/theta from the group's box).  Partial
// sums (about 32 interactions per slot) are folded into a (hi, lo) pair by
// TwoSum.  Variant 1 is the naive form: absolute FP32 coordinates and plain
// sums.  A body is never paired with itself: particle tiles that hold bodies
// of the walking group (a ballot tells) run a loop that skips equal indices;
// all other tiles run the plain loop.  With eps = 0 zero distances are
// skipped as well.
#include <cuda_runtime.h>

#include "bh_internal.cuh"

namespace bh {
namespace {

struct WarpSmem {
  int clist[64];
  int plist[64];
  // staged cells: (dx, dy, dz, M), (Qxx, Qyy, Qzz, Qxy), (Qxz, Qyz, 0, 0); entries >= 32 stay null
  float4 sc[64][3];
  // staged bodies: (S_hi, m), (S_lo, 0) -- offsets from the group centre as two floats;
  // reused for the per-slot partial sums when a group ends (then re-nulled)
  float4 sp[64][2];
  int pidx[64];  // their sorted indices (read only for tiles holding the group's own bodies)
  float box[6];  // group bounding box (min xyz, max xyz), offsets from the centre
  float ctr[3];  // group centre
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
constexpr int kWalkThreads = 128;  // 4 warps per block
constexpr int kWalkMinBlocks = 5;  // 20 resident warps per SM (96 registers)

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

// a - b rounded, and the exact rounding error of that subtraction (Knuth's TwoSum).
__device__ __forceinline__ float two_diff(float a, float b, float &err) {
  float s = a - b;
  float bb = s - a;
  err = (a - (s - bb)) - (b + bb);
  return s;
}

template <int VAR>
__device__ __forceinline__ void fold(Acc &hi, Acc &lo, Acc &t) {
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
  t = Acc{0.f, 0.f, 0.f, 0.f};
}

struct Target {
  float hx, hy, hz;  // offset from the group centre, rounded
  float lx, ly, lz;  // its residual (variant 0) so that hi + lo is the offset to ~2^-48
};

// Softened particle-particle interaction of a staged source (S_hi, m), S_lo on
// a target: 20 flops by the convention FMA = 2, rsqrt = 1 (the two-float
// difference d = (S_hi - T_hi) + (S_lo - T_lo) costs 6 more: its first term is
// exact for close pairs, so a pair keeps its relative accuracy however far it
// is from the group centre).  SELF: skip the pair of a body with itself (same
// index); GUARD: eps = 0, zero distances skipped.
template <int VAR, bool GUARD, bool SELF>
__device__ __forceinline__ void pp(Acc &a, const Target &t, const float4 sh, const float4 sl, float eps2,
                                   int me = 0, int other = 1) {
  float dx, dy, dz;
  if (VAR == 0) {
    dx = (sh.x - t.hx) + (sl.x - t.lx);
    dy = (sh.y - t.hy) + (sl.y - t.ly);
    dz = (sh.z - t.hz) + (sl.z - t.lz);
  } else {
    dx = sh.x - t.hx;
    dy = sh.y - t.hy;
    dz = sh.z - t.hz;
  }
  float r2 = fmaf(dx, dx, eps2);
  r2 = fmaf(dy, dy, r2);
  r2 = fmaf(dz, dz, r2);
  float ri = rsqrtf(r2);
  if (GUARD) ri = (r2 > 0.f) ? ri : 0.f;
  if (SELF) ri = (me == other) ? 0.f : ri;
  float mr = sh.w * ri;
  float mr3 = mr * ri * ri;
  a.p -= mr;
  a.x = fmaf(mr3, dx, a.x);
  a.y = fmaf(mr3, dy, a.y);
  a.z = fmaf(mr3, dz, a.z);
}

// Softened particle-cell interaction, monopole + quadrupole, with d = com -
// target: a = M d/s^3 - Q d/s^5 + (5/2)(d.Q.d) d/s^7, phi = -M/s - (d.Q.d)/(2 s^5).
// 54 flops by the convention above.
__device__ __forceinline__ void pc(Acc &a, const Target &t, const float4 c0, const float4 q0, const float4 q1,
                                   float eps2) {
  float dx = c0.x - t.hx, dy = c0.y - t.hy, dz = c0.z - t.hz;
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

template <int VAR>
__device__ __forceinline__ Target make_target(float4 h, float4 l, float cx, float cy, float cz) {
  Target t;
  if (VAR == 0) {
    float ex, ey, ez;
    t.hx = two_diff(h.x, cx, ex);
    t.hy = two_diff(h.y, cy, ey);
    t.hz = two_diff(h.z, cz, ez);
    t.lx = ex + l.x;
    t.ly = ey + l.y;
    t.lz = ez + l.z;
  } else {
    t.hx = h.x;
    t.hy = h.y;
    t.hz = h.z;
    t.lx = t.ly = t.lz = 0.f;
  }
  return t;
}

template <int VAR, bool GUARD, int MODE>
__global__ void __launch_bounds__(kWalkThreads, kWalkMinBlocks) k_walk(WalkArgs A) {
  extern __shared__ WarpSmem s_warp[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  WarpSmem &S = s_warp[wib];
  const size_t gw = (size_t)blockIdx.x * (blockDim.x >> 5) + wib;
  int *cur = A.stack + gw * 2 * (size_t)A.cap;
  int *nxt = cur + A.cap;
  const unsigned lt = lanemask_lt();
  const float eps2 = A.eps2;
  const float4 null_src = make_float4(kFar, kFar, kFar, 0.f);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // entries 32..63 of the staging arrays are permanent nulls (zero mass, far away)
  S.sc[32 + lane][0] = null_src;
  S.sc[32 + lane][1] = zero4;
  S.sc[32 + lane][2] = zero4;
  S.sp[32 + lane][0] = null_src;
  S.sp[32 + lane][1] = zero4;
  S.pidx[32 + lane] = -1;
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
    // slots: a group of n bodies gets k = floor(64/n) slots per body (one for
    // n > 32); slot s holds body s % n and takes the sources j = s / n (mod k)
    const int k = (n > 32) ? 1 : min(64 / n, 32);
    int b0, b1, ph0, ph1;
    bool v0, v1;
    if (k == 1) {
      b0 = lane;
      b1 = lane + 32;
      ph0 = ph1 = 0;
      v0 = b0 < n;
      v1 = b1 < n;
    } else {
      const int ns = n * k;
      v0 = lane < ns;
      v1 = lane + 32 < ns;
      b0 = lane % n;
      b1 = (lane + 32) % n;
      ph0 = v0 ? lane / n : 0;
      ph1 = v1 ? (lane + 32) / n : 0;
    }
    // group centre (a float: the first body) and the slots' targets
    float cx = 0.f, cy = 0.f, cz = 0.f;
    if (VAR == 0) {
      float4 c = A.part_hi[gb];
      cx = c.x;
      cy = c.y;
      cz = c.z;
    }
    const int lb0 = gb + min(b0, n - 1), lb1 = gb + min(b1, n - 1);
    const Target T0 = make_target<VAR>(A.part_hi[lb0], A.part_lo[lb0], cx, cy, cz);
    const Target T1 = make_target<VAR>(A.part_hi[lb1], A.part_lo[lb1], cx, cy, cz);
    // tight bounding box of the group's bodies
    float bminx = fminf(v0 ? T0.hx : INFINITY, v1 ? T1.hx : INFINITY);
    float bminy = fminf(v0 ? T0.hy : INFINITY, v1 ? T1.hy : INFINITY);
    float bminz = fminf(v0 ? T0.hz : INFINITY, v1 ? T1.hz : INFINITY);
    float bmaxx = fmaxf(v0 ? T0.hx : -INFINITY, v1 ? T1.hx : -INFINITY);
    float bmaxy = fmaxf(v0 ? T0.hy : -INFINITY, v1 ? T1.hy : -INFINITY);
    float bmaxz = fmaxf(v0 ? T0.hz : -INFINITY, v1 ? T1.hz : -INFINITY);
    for (int o = 16; o > 0; o >>= 1) {
      bminx = fminf(bminx, __shfl_xor_sync(kFull, bminx, o));
      bminy = fminf(bminy, __shfl_xor_sync(kFull, bminy, o));
      bminz = fminf(bminz, __shfl_xor_sync(kFull, bminz, o));
      bmaxx = fmaxf(bmaxx, __shfl_xor_sync(kFull, bmaxx, o));
      bmaxy = fmaxf(bmaxy, __shfl_xor_sync(kFull, bmaxy, o));
      bmaxz = fmaxf(bmaxz, __shfl_xor_sync(kFull, bmaxz, o));
    }
    if (lane == 0) {
      S.box[0] = bminx;
      S.box[1] = bminy;
      S.box[2] = bminz;
      S.box[3] = bmaxx;
      S.box[4] = bmaxy;
      S.box[5] = bmaxz;
      S.ctr[0] = cx;
      S.ctr[1] = cy;
      S.ctr[2] = cz;
    }
    __syncwarp();
    Acc h0 = {0, 0, 0, 0}, l0 = {0, 0, 0, 0}, h1 = {0, 0, 0, 0}, l1 = {0, 0, 0, 0};
    Acc t0 = {0, 0, 0, 0}, t1 = {0, 0, 0, 0};  // partial sums since the last fold
    int since = 0;                              // interactions per slot since the last fold
    int cn = 0, pn = 0, ncell = 0, npart = 0;
    unsigned long long csum = 0, psum = 0;

    auto after_tile = [&](int cnt) {
      since += (cnt + k - 1) / k;
      if (since >= 32) {
        fold<VAR>(h0, l0, t0);
        fold<VAR>(h1, l1, t1);
        since = 0;
      }
    };

    // ---- evaluate the first `cnt` entries of the cell list
    auto eval_cells = [&](int cnt) {
      if (lane < cnt) {
        int cc = S.clist[lane];
        float4 a = A.mom[4 * (size_t)cc], b = A.mom[4 * (size_t)cc + 1];
        float4 q0 = A.mom[4 * (size_t)cc + 2], q1 = A.mom[4 * (size_t)cc + 3];
        float dx, dy, dz;
        if (VAR == 0) {
          dx = (a.x - S.ctr[0]) + b.x;
          dy = (a.y - S.ctr[1]) + b.y;
          dz = (a.z - S.ctr[2]) + b.z;
        } else {
          dx = a.x;
          dy = a.y;
          dz = a.z;
        }
        S.sc[lane][0] = make_float4(dx, dy, dz, a.w);
        S.sc[lane][1] = q0;
        S.sc[lane][2] = make_float4(q1.x, q1.y, 0.f, 0.f);
      } else {
        S.sc[lane][0] = null_src;
        S.sc[lane][1] = zero4;
        S.sc[lane][2] = zero4;
      }
      __syncwarp();
      if (k == 1) {
#pragma unroll 1
        for (int j = 0; j < cnt; ++j) {
          const float4 c0 = S.sc[j][0], q0 = S.sc[j][1], q1 = S.sc[j][2];
          pc(t0, T0, c0, q0, q1, eps2);
          pc(t1, T1, c0, q0, q1, eps2);
        }
      } else {
#pragma unroll 1
        for (int j = 0; j < cnt; j += k) {
          pc(t0, T0, S.sc[j + ph0][0], S.sc[j + ph0][1], S.sc[j + ph0][2], eps2);
          pc(t1, T1, S.sc[j + ph1][0], S.sc[j + ph1][1], S.sc[j + ph1][2], eps2);
        }
      }
      after_tile(cnt);
      __syncwarp();
    };

    // ---- evaluate the first `cnt` entries of the particle list
    auto eval_bodies = [&](int cnt) {
      bool member = false;
      if (lane < cnt) {
        int b = S.plist[lane];
        member = (unsigned)(b - gb) < (unsigned)n;
        const Target s = make_target<VAR>(A.part_hi[b], A.part_lo[b], S.ctr[0], S.ctr[1], S.ctr[2]);
        S.sp[lane][0] = make_float4(s.hx, s.hy, s.hz, A.part_hi[b].w);
        S.sp[lane][1] = make_float4(s.lx, s.ly, s.lz, 0.f);
        S.pidx[lane] = b;
      } else {
        S.sp[lane][0] = null_src;
        S.sp[lane][1] = zero4;
        S.pidx[lane] = -1;
      }
      const bool self_tile = __any_sync(kFull, member);
      __syncwarp();
      if (self_tile) {
        // a tile with the group's own bodies: skip each body's pair with itself by index
        const int me0 = gb + b0, me1 = gb + b1;
        for (int j = 0; j < cnt; j += k) {
          pp<VAR, GUARD, true>(t0, T0, S.sp[j + ph0][0], S.sp[j + ph0][1], eps2, me0, S.pidx[j + ph0]);
          pp<VAR, GUARD, true>(t1, T1, S.sp[j + ph1][0], S.sp[j + ph1][1], eps2, me1, S.pidx[j + ph1]);
        }
      } else if (k == 1) {
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
          const float4 sh = S.sp[j][0], sl = S.sp[j][1];
          pp<VAR, GUARD, false>(t0, T0, sh, sl, eps2);
          pp<VAR, GUARD, false>(t1, T1, sh, sl, eps2);
        }
      } else {
#pragma unroll 2
        for (int j = 0; j < cnt; j += k) {
          pp<VAR, GUARD, false>(t0, T0, S.sp[j + ph0][0], S.sp[j + ph0][1], eps2);
          pp<VAR, GUARD, false>(t1, T1, S.sp[j + ph1][0], S.sp[j + ph1][1], eps2);
        }
      }
      after_tile(cnt);
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
        float rx = m.x - S.ctr[0], ry = m.y - S.ctr[1], rz = m.z - S.ctr[2];
        float ex = fmaxf(fmaxf(S.box[0] - rx, rx - S.box[3]), 0.f);
        float ey = fmaxf(fmaxf(S.box[1] - ry, ry - S.box[4]), 0.f);
        float ez = fmaxf(fmaxf(S.box[2] - rz, rz - S.box[5]), 0.f);
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
          int kk = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            int v = __shfl_sync(kFull, pin, kk + step - 1);
            if (v <= si) kk += step;
          }
          const int of = __shfl_sync(kFull, lk.x, kk);
          const int oe = __shfl_sync(kFull, pex, kk);
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
    fold<VAR>(h0, l0, t0);
    fold<VAR>(h1, l1, t1);

    // ---- combine the slots of each body and write
    auto write_body = [&](int b, float ox, float oy, float oz, float op) {
      const int gi = gb + b;
      if (MODE == kOutSorted) {
        A.acc_sorted[gi] = make_float4(ox, oy, oz, op);
      } else {
        const size_t j = A.perm[gi];
        A.acc_out[3 * j] = ox;
        A.acc_out[3 * j + 1] = oy;
        A.acc_out[3 * j + 2] = oz;
        A.pot_out[j] = op;
      }
    };
    if (k == 1) {
      if (v0) write_body(b0, h0.x + l0.x, h0.y + l0.y, h0.z + l0.z, h0.p + l0.p);
      if (v1) write_body(b1, h1.x + l1.x, h1.y + l1.y, h1.z + l1.z, h1.p + l1.p);
    } else {
      // slot s -> sp[s] = (hi), (lo); body b sums slots b, b + n, ..., b + n (k - 1)
      S.sp[lane][0] = make_float4(h0.x, h0.y, h0.z, h0.p);
      S.sp[lane][1] = make_float4(l0.x, l0.y, l0.z, l0.p);
      S.sp[32 + lane][0] = make_float4(h1.x, h1.y, h1.z, h1.p);
      S.sp[32 + lane][1] = make_float4(l1.x, l1.y, l1.z, l1.p);
      __syncwarp();
      if (lane < n) {
        float4 H = S.sp[lane][0], L = S.sp[lane][1];
        for (int q = 1; q < k; ++q) {
          const float4 h = S.sp[lane + q * n][0], l = S.sp[lane + q * n][1];
          two_sum_into(H.x, L.x, h.x);
          two_sum_into(H.y, L.y, h.y);
          two_sum_into(H.z, L.z, h.z);
          two_sum_into(H.w, L.w, h.w);
          L.x += l.x;
          L.y += l.y;
          L.z += l.z;
          L.w += l.w;
        }
        write_body(lane, H.x + L.x, H.y + L.y, H.z + L.z, H.w + L.w);
      }
      __syncwarp();
      S.sp[32 + lane][0] = null_src;
      S.sp[32 + lane][1] = zero4;
      __syncwarp();
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
