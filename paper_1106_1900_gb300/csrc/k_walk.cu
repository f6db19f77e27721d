// k_walk.cu -- the breadth-first group walk and force evaluation (§2.2, §3.3).
//
// The paper walks and evaluates in one kernel: a group's interaction lists
// fill shared memory and are evaluated whenever they are full, the rest when
// the walk ends.  Here one warp does a group at a time: walk_some walks the
// tree, appending to two bounded list buffers of the warp (cells, bodies;
// global memory, L2-resident), and eval_lists sums the buffered lists tile
// by tile.  The default kernel runs both per group:
//
//  k_size_hist, k_order   place the groups by size, largest first (the cost
//              of a group is not known before its walk).
//  k_walk      persistent warps take groups from a counter in that order and
//              walk each.  When the walk ends, the lists are evaluated
//              straight from the buffers; when a buffer would overflow first
//              (list_buffer entries), the walk pauses (its state saved in the
//              warp's scratch), both buffers' whole tiles are evaluated, the
//              rest moves to their fronts and the walk goes on.  No list
//              length is limited, no list pool exists, and other warps'
//              arithmetic runs while a warp walks.
//
// The split form (walk_split = 1; the FP64 evaluation variant always) runs
// the two as separate persistent kernels on whole lists:
//
//  k_traverse  one warp per group (groups taken from a counter).  The current
//              level of the walk is read 32 cells at a time from a per-warp
//              stack in global memory; each lane applies Eq. 1 to one cell
//              (d^2 > (l/theta + delta)^2, d = distance from the cell's centre
//              of mass to the group's bounding box).  Accepted cells go to the
//              cell list, opened nodes push their (contiguous) children on the
//              next level's stack, opened leaves append their (contiguous)
//              bodies to the particle list; appends are warp ballots and warp
//              prefix sums.  The lists are written to per-warp scratch, then
//              copied into one pool at an exact offset (one atomic per group).
//  k_order     sorts the groups by their estimated evaluation cost (a
//              logarithmic histogram filled by k_traverse, one scatter).
//  k_eval      one warp per group, most expensive first, so that the launch
//              ends on cheap groups.  Lists are summed 64 entries at a time:
//              each lane gathers and stages two into shared memory, then every
//              lane sums the tile from there.
// The two forms build the same lists; with buffers at least as long as
// every list they also sum them in the same order (identical results).
//
// Slots: every lane holds two target slots, 64 per warp.  A group of n <= 32
// bodies is laid out with h = ceil(n/2): lane l holds bodies l mod h and
// l mod h + h in phase l div h, so k = floor(32/h) slots per body, each taking
// every k-th source from its phase on, summed per body when the group ends --
// the paper's "several threads per particle" for small groups, generalised so
// that few slots idle.  A group of n > 32 bodies has one slot per body.  Both
// slots of a lane read the same source, so the arithmetic runs on packed FP32
// pairs (f32x2 FMA, add, multiply: one instruction for both slots, half the
// issue slots of scalar code at the same FP32 rate); a staged value is read
// once and paired with itself in registers.  A group of
// 33..48 bodies would idle a quarter of the slots or more; it is evaluated in
// two or three passes over the same lists, each for a subset of its bodies
// small enough for three or four slots per body (eval_passes).
//
// Precision (variant 0): coordinates are offsets from the group centre c (a
// float: the first body's position), each kept as two floats -- the
// difference of the high parts and the rest, hi + lo the offset to ~2^-48 --
// built from the two-float body positions.  Particle-particle terms
// difference both parts, so a close pair stays accurate however far from c it
// lies; particle-cell terms use the high part, which is off by at most the
// body's low part (2^-25 of its coordinate), far below l/theta for any cell
// of a 20-level tree.  Keys deeper than 20 levels take variant 3: the high
// part is the correctly rounded offset and the opening test also reads the
// low part of each cell's position (a level-30 cell is 2^-30 L).  Partial
// sums (about 64 interactions per slot) are folded into a (hi, lo) pair by
// TwoSum.  Variant 1 is the naive form: absolute FP32 coordinates and plain
// sums.  A body is never paired with itself: particle tiles that hold bodies
// of the walking group (a ballot tells) run a loop that skips equal indices;
// all other tiles run the plain loop.  With eps = 0 zero distances are
// skipped as well.
#include <cuda_runtime.h>

#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr float kFar = 1e18f;
constexpr int kWarps = 4;  // warps per block of both kernels
constexpr int kThreads = 32 * kWarps;
constexpr int kEvalMinBlocks = 6;
constexpr int kWalkMinBlocks = 6;  // the fused walk (7 measured slower at N_crit = 96)
// Lists are summed in tiles of kTile entries, each lane staging two.  With k
// phases a lane reads entries ph, ph + k, ... < cnt + ph, the last one at
// most k ceil(64 / k) - 1, and k = 32 / h is one of 1, 2, 3, 4, 5, 6, 8, 10,
// 16, 32: at most entry 69 (k = 10); entries 64..kStage-1 are permanent nulls.
constexpr int kTile = 64;
constexpr int kStage = 72;
static_assert(kTile % 32 == 0 && kStage >= kTile + 6, "staging: whole warps per tile, nulls up to entry 69");
// Interactions per slot between folds of the FP32 partial sums into the
// compensated (hi, lo) pair: 64 (32 measured 1.5 % slower; a plain FP32 sum
// of 64 terms is off by ~sqrt(64) ulp of its terms' magnitude, typically).
constexpr int kFoldEvery = 64;
// Ints of list scratch per warp of the fused walk: a cell buffer and a body
// buffer of cap entries each (cap a multiple of 64), then 32 waiting leaves
// (int2), then the walk's state (kWalkStateInts; global memory, L1-cached:
// shared memory is kept to what six blocks of the walk need per SM, which
// leaves the L1 cache its size).
constexpr int kWalkStateInts = 32;
__host__ __device__ constexpr long walk_stride(int cap) { return 2L * cap + 64 + kWalkStateInts; }

// Arithmetic variants: 0 group-relative FP32 with compensated tiles, 1 naive
// FP32; 3 is variant 0 for keys deeper than 20 levels, whose cells can be
// smaller than the float spacing at their position: offsets from the group
// centre are rounded once from the whole two-float difference, and the
// opening test adds the low part of each record's position.
constexpr int kVarDeep = 3;
__host__ __device__ constexpr bool relative(int var) { return var == 0 || var == kVarDeep; }

struct Target {
  float hx, hy, hz;  // offset from the group centre, rounded
  float lx, ly, lz;  // its residual (variant 0) so that hi + lo is the offset to ~2^-48
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

// Slot layout of a (sub)group of n <= 64 bodies on a warp's 64 slots: lane l
// holds bodies b = l mod h and b + h (h = pair_stride(n)) in phase l div h, so
// both slots of a lane read the same source; a body gets 32 / h slots.
__host__ __device__ constexpr int pair_stride(int n) { return (n > 32) ? 32 : ((n + 1) >> 1 > 1 ? (n + 1) >> 1 : 1); }
__host__ __device__ constexpr int slots_per_body(int n) { return 32 / pair_stride(n); }

// Passes over a group's lists.  A warp holds at most 64 targets, so a group
// of n > 64 bodies needs at least ceil(n / 64) passes; a group of 33..63
// bodies gets one slot per body and leaves 64 - n slots idle.  P passes over
// subsets of ceil(n / P) bodies each, all on the group's own lists (a list
// valid for a group is valid for any subset of it), fill the slots better.  A
// pass costs ceil(32 / k) iterations per 32 list entries, but no less than ~8:
// below that the tile's gather from L2 is no longer hidden behind its
// arithmetic, and every pass re-gathers the lists.  So groups of up to 32
// bodies keep one pass, 33..42 bodies take two, 43..48 three.  The rule is
// tabulated for n = 0..kMaxCrit at compile time (c_passes).
__host__ __device__ constexpr int passes_rule(int n) {
  if (n <= 32) return 1;
  const int p0 = (n + 63) / 64;
  int best = p0, best_cost = 1 << 30;
  for (int P = p0; P <= p0 + 3; ++P) {
    const int nb = (n + P - 1) / P;
    const int k = slots_per_body(nb);
    const int it = (32 + k - 1) / k;
    const int cost = P * ((it > 8 ? it : 8) + 1);
    if (cost < best_cost) {
      best_cost = cost;
      best = P;
    }
  }
  const int nb = (n + best - 1) / best;
  return (n + nb - 1) / nb;  // no empty last pass
}

struct PassTable {
  uint8_t p[kMaxCrit + 1];
  constexpr PassTable() : p() {
    for (int n = 0; n <= kMaxCrit; ++n) p[n] = (uint8_t)passes_rule(n);
  }
};
__constant__ PassTable c_passes = PassTable();

__device__ __forceinline__ int eval_passes(int n) { return c_passes.p[min(max(n, 0), kMaxCrit)]; }

// Logarithmic bucket of an estimated cost w >= 1: eight buckets per octave,
// increasing with w, below kCostBuckets for any int.
__device__ __forceinline__ int cost_bucket(int w) {
  const unsigned u = (unsigned)max(w, 1);
  const int msb = 31 - __clz(u);
  const unsigned frac = (msb >= 3) ? (u >> (msb - 3)) & 7u : (u << (3 - msb)) & 7u;
  return 8 * msb + (int)frac;
}

// Offset of a two-float coordinate (h, l) from the float c: the difference of
// the high parts (exact with its rounding error) plus the low part, rounded
// once (hi) with the exact residual (lo).  The rounded offset is what the
// opening test and the particle-cell terms read; it must be the correctly
// rounded one, since the low part of a coordinate can exceed the size of the
// smallest cells (keys deeper than 20 levels: cells of 6e-8 at 0.3, whose
// float spacing is 3e-8).
__device__ __forceinline__ void rounded_offset(float h, float l, float c, float &hi, float &lo) {
  float e;
  const float d = two_diff(h, c, e);  // d + e = h - c
  const float r = e + l;              // |r| <= ulp(h): its rounding is below 2^-47 |h|
  const float s = d + r;
  const float bb = s - d;
  lo = (d - (s - bb)) + (r - bb);  // TwoSum: s + lo = d + r
  hi = s;
}

template <int VAR>
__device__ __forceinline__ Target make_target(float4 h, float4 l, float cx, float cy, float cz) {
  Target t;
  if (VAR == kVarDeep) {
    rounded_offset(h.x, l.x, cx, t.hx, t.lx);
    rounded_offset(h.y, l.y, cy, t.hy, t.ly);
    rounded_offset(h.z, l.z, cz, t.hz, t.lz);
  } else if (VAR == 0) {  // the difference of the high parts and the rest: enough where cells exceed 2^-20 L
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

// ================================================================ traversal
struct TravArgs {
  const float4 *__restrict__ part_hi;
  const float4 *__restrict__ part_lo;
  const float4 *__restrict__ mac;
  const float4 *__restrict__ mac_lo;  // keys deeper than 20 levels: the low parts of the records' positions
  const int2 *__restrict__ link;
  const int32_t *__restrict__ g_beg;
  const int32_t *__restrict__ g_sys;
  const int32_t *__restrict__ sys_root;
  const int32_t *__restrict__ counts;
  int32_t *stack;
  int cap;
  int32_t *scratch;  // per warp: list_cap cells, then list_cap bodies
  int list_cap;      // entries of each list (fused walk: its buffers; split walk: a group's whole lists)
  uint32_t *pool;
  unsigned long long pool_cap;
  unsigned long long *pool_ctr;
  int4 *g_list;  // per group: {pool offset / kPoolAlign, cells, bodies, estimated evaluation cost}
  uint32_t *work_hist;  // groups per cost bucket
  int box_mac;           // 1: minimal-distance criterion (mac record = cube centre, half side)
  float two_over_theta;  // its l/theta = (l/2) (2/theta)
  int n;
  uint32_t *queue;
  int32_t *g_npc;
  int32_t *g_npp;
  unsigned long long *g_csum;
  unsigned long long *g_psum;
  unsigned long long *totals;
  int32_t *status;
};

// dst[0..cnt) = src[0..cnt), a warp, four independent loads in flight per lane
__device__ __forceinline__ void copy_list(uint32_t *__restrict__ dst, const int *__restrict__ src, int cnt,
                                          int lane) {
  for (int i0 = 0; i0 < cnt; i0 += 128) {
    int v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 32 * u + lane;
      v[u] = (i < cnt) ? src[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 32 * u + lane;
      if (i < cnt) dst[i] = (uint32_t)v[u];
    }
  }
}

// State of one group's breadth-first walk between two calls of walk_some: a
// register copy in every lane of the warp (the same values), which the fused
// walk saves to its scratch while it evaluates full buffers.
struct __align__(16) WalkState {
  float box[6];  // the group's tight bounding box (offsets from its centre c)
  float c[3];    // the group's centre: its first body
  int depth;     // levels of the walk so far
  int ncur;      // cells of the current level (on the stack selected by flip)
  int nnext;     // cells pushed for the next level
  int base;      // next chunk of the current level
  int flip;      // 0: the current level is on stack `cur`, 1: on `nxt`
  int mid;       // 1: the walk stopped inside a level (at chunk `base`)
  int bc;        // cells in the cell list (buffer)
  int bp;        // bodies in the particle list (buffer)
  int ncell;     // whole cell-list length
  int npart;     // whole particle-list length (bodies)
  int npend;     // opened leaves of the last chunk whose bodies are not all listed yet (in pend[])
  int pend_tot;  // their bodies
  int pend_done; // of which listed
  int g;         // fused walk: the group (-1: none)
  int parts;     // fused walk: evaluations of the group's buffers so far
  unsigned long long csum, psum;  // sums of the listed cell and body indices
};

static_assert(sizeof(WalkState) <= 4 * kWalkStateInts, "the walk state fits its scratch slot");

// Group g's walk starts: centre, tight bounding box, the root on stack cur.
template <int VAR>
__device__ __forceinline__ void walk_start(const TravArgs &A, WalkState &W, int g, int lane, int *cur) {
  const int gb = A.g_beg[g];
  const int n = A.g_beg[g + 1] - gb;
  // group centre and tight bounding box (offsets from the centre, rounded)
  float cx = 0.f, cy = 0.f, cz = 0.f;
  if (relative(VAR)) {
    const float4 c = A.part_hi[gb];
    cx = c.x;
    cy = c.y;
    cz = c.z;
  }
  float bminx = INFINITY, bminy = INFINITY, bminz = INFINITY;
  float bmaxx = -INFINITY, bmaxy = -INFINITY, bmaxz = -INFINITY;
  for (int b = lane; b < n; b += 32) {
    const Target t = make_target<VAR>(A.part_hi[gb + b], A.part_lo[gb + b], cx, cy, cz);
    bminx = fminf(bminx, t.hx);
    bminy = fminf(bminy, t.hy);
    bminz = fminf(bminz, t.hz);
    bmaxx = fmaxf(bmaxx, t.hx);
    bmaxy = fmaxf(bmaxy, t.hy);
    bmaxz = fmaxf(bmaxz, t.hz);
  }
  for (int o = 16; o > 0; o >>= 1) {
    bminx = fminf(bminx, __shfl_xor_sync(kFull, bminx, o));
    bminy = fminf(bminy, __shfl_xor_sync(kFull, bminy, o));
    bminz = fminf(bminz, __shfl_xor_sync(kFull, bminz, o));
    bmaxx = fmaxf(bmaxx, __shfl_xor_sync(kFull, bmaxx, o));
    bmaxy = fmaxf(bmaxy, __shfl_xor_sync(kFull, bmaxy, o));
    bmaxz = fmaxf(bmaxz, __shfl_xor_sync(kFull, bmaxz, o));
  }
  // every lane holds the state (a register copy, uniform across the warp)
  W.box[0] = bminx;
  W.box[1] = bminy;
  W.box[2] = bminz;
  W.box[3] = bmaxx;
  W.box[4] = bmaxy;
  W.box[5] = bmaxz;
  W.c[0] = cx;
  W.c[1] = cy;
  W.c[2] = cz;
  W.depth = 0;
  W.ncur = 1;
  W.nnext = 0;
  W.base = 0;
  W.flip = 0;
  W.mid = 0;
  W.bc = W.bp = 0;
  W.ncell = W.npart = 0;
  W.npend = W.pend_tot = W.pend_done = 0;
  W.csum = W.psum = 0ull;
  if (lane == 0) cur[0] = A.sys_root[A.g_sys[g]];
  __syncwarp();
}

// The bodies at positions done + lane of the opened leaves (first body of
// leaf j = first_j, inclusive prefix of the counts = pin_j, held by lane j):
// the leaf of each position is found by a binary search of the prefix sums
// spread over the warp.  -1 past tot.
__device__ __forceinline__ int leaf_body(int pin, int first, int pex, int done, int tot, int lane) {
  const int si = done + lane;
  int kk = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int v = __shfl_sync(kFull, pin, kk + step - 1);
    if (v <= si) kk += step;
  }
  const int of = __shfl_sync(kFull, first, kk);
  const int oe = __shfl_sync(kFull, pex, kk);
  return (si < tot) ? of + (si - oe) : -1;
}

// The breadth-first walk of §2.2 by one warp, from the state in W until it
// ends (returns true) or, FUSED, until a buffer of list_cap entries is full
// (returns false: the caller evaluates the buffers' whole tiles and calls
// again).  Each lane applies the opening test (Eq. 1, or the
// minimal-distance criterion) to one cell of a chunk of 32: accepted cells go
// to the cell list cl, opened nodes push their (contiguous) children on the
// next level's stack, opened leaves append their (contiguous) bodies to the
// particle list pl; appends are warp ballots and prefix sums.  FUSED: a chunk
// is started only if its accepted cells fit; the bodies of its opened leaves
// go straight to the list if they fit, else the leaves wait (up to 32, right
// after pl's cap entries, see list_waiting) and the walk stops.  Without
// FUSED the lists are the group's whole lists: entries past list_cap are
// counted but not stored.
template <int VAR, bool FUSED>
__device__ __forceinline__ bool walk_some(const TravArgs &A, WalkState &W, int lane, unsigned lt, int *cur, int *nxt,
                                          int *cl, int *pl) {
  const int cap = A.list_cap;
  const float bminx = W.box[0], bminy = W.box[1], bminz = W.box[2];
  const float bmaxx = W.box[3], bmaxy = W.box[4], bmaxz = W.box[5];
  const float cx = W.c[0], cy = W.c[1], cz = W.c[2];
  int depth = W.depth, ncur = W.ncur, nnext = W.nnext, base = W.base;
  int bc = W.bc, bp = W.bp, ncell = W.ncell, npart = W.npart;
  int flip = W.flip;
  int *cstk = flip ? nxt : cur, *nstk = flip ? cur : nxt;
  bool mid = W.mid != 0;  // resuming inside a level
  // per-lane partial sums of the listed indices, lane 0 starting from the totals so far
  unsigned long long csum = (lane == 0) ? W.csum : 0ull, psum = (lane == 0) ? W.psum : 0ull;
  bool full = false;
  while (!full && ncur > 0) {
    if (!mid) {  // a new level
      if (++depth > kLevelsMax + 1) {  // a tree has at most D + 1 <= 31 levels: never loop on a corrupt one
        if (lane == 0) set_status(A.status, BH_ERR_STATE);
        ncur = 0;
        break;
      }
      nnext = 0;
      base = 0;
    }
    mid = false;
    // the frontier is read 32 cells at a time; the next chunk's loads are
    // issued before this chunk is processed (software pipelining)
    int ci_n = 0;
    float4 m_n = make_float4(0.f, 0.f, 0.f, 0.f);
    int2 lk_n = make_int2(0, 0);
    if (base + lane < ncur) {
      ci_n = cstk[base + lane];
      m_n = A.mac[ci_n];
      lk_n = A.link[ci_n];
    }
    int ci_nn = (base + 32 + lane < ncur) ? cstk[base + 32 + lane] : 0;  // stack entries run a chunk further ahead
    for (; base < ncur; base += 32) {
      if (FUSED && bc + 32 > cap) {  // this chunk's cells could overflow the buffer: evaluate first
        full = true;
        break;
      }
      const bool have = base + lane < ncur;
      const int ci = ci_n;
      const float4 m = m_n;
      const int2 lk = lk_n;
      if (base + 32 + lane < ncur) {
        ci_n = ci_nn;
        m_n = A.mac[ci_n];
        lk_n = A.link[ci_n];
      }
      if (base + 64 + lane < ncur) ci_nn = cstk[base + 64 + lane];
      float rx = m.x - cx, ry = m.y - cy, rz = m.z - cz;
      if (VAR == kVarDeep && have) {  // cells below level 20 can be smaller than the float spacing at their position
        const float4 ml = A.mac_lo[ci];
        rx += ml.x;
        ry += ml.y;
        rz += ml.z;
      }
      float ex, ey, ez, ro;
      if (!A.box_mac) {  // Eq. 1: the centre of mass's distance to the box against r_open = m.w
        ex = fmaxf(fmaxf(bminx - rx, rx - bmaxx), 0.f);
        ey = fmaxf(fmaxf(bminy - ry, ry - bmaxy), 0.f);
        ez = fmaxf(fmaxf(bminz - rz, rz - bmaxz), 0.f);
        ro = m.w;
      } else {  // minimal distance: the gap between the cube (half side m.w) and the box against l/theta
        ex = fmaxf(fmaxf(bminx - rx, rx - bmaxx) - m.w, 0.f);
        ey = fmaxf(fmaxf(bminy - ry, ry - bmaxy) - m.w, 0.f);
        ez = fmaxf(fmaxf(bminz - rz, rz - bmaxz) - m.w, 0.f);
        ro = m.w * A.two_over_theta;
      }
      const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      const bool accept = have && d2 > ro * ro;
      const bool open = have && !accept;
      const bool leaf = lk.y < 0;
      // accepted cells -> cell list
      const unsigned ab = __ballot_sync(kFull, accept);
      if (accept) {
        const int at = bc + __popc(ab & lt);
        if (at < cap) cl[at] = ci;
        csum += (unsigned long long)ci;
      }
      ncell += __popc(ab);
      bc += __popc(ab);
      // opened nodes -> children on the next level, opened leaves -> bodies
      const int nch = (open && !leaf) ? min(max(lk.y, 0), 8) : 0;
      const int np = (open && leaf) ? (lk.y & 0x7fffffff) : 0;
      int inc, pin, tot, ptot;
      if (__all_sync(kFull, np < (1 << 17))) {
        // both prefix sums in one scan: children (<= 256 a chunk) in the low
        // 10 bits, bodies (< 2^22 a chunk) above them
        unsigned v = (unsigned)nch | ((unsigned)np << 10);
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(kFull, v, o);
          if (lane >= o) v += y;
        }
        const unsigned vt = __shfl_sync(kFull, v, 31);
        inc = (int)(v & 1023u);
        pin = (int)(v >> 10);
        tot = (int)(vt & 1023u);
        ptot = (int)(vt >> 10);
      } else {  // a leaf of 2^17 bodies or more (coincident positions): two scans
        inc = nch;
        pin = np;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, inc, o);
          const int z = __shfl_up_sync(kFull, pin, o);
          if (lane >= o) {
            inc += y;
            pin += z;
          }
        }
        tot = __shfl_sync(kFull, inc, 31);
        ptot = __shfl_sync(kFull, pin, 31);
      }
      if (nnext + tot <= A.cap) {
        int *dst = nstk + (nnext + inc - nch);
#pragma unroll
        for (int j = 0; j < 8; ++j)  // predicated stores, no divergent loop
          if (j < nch) dst[j] = lk.x + j;
        nnext += tot;
      } else if (tot > 0) {
        if (lane == 0) set_status(A.status, BH_ERR_CAPACITY);
      }
      // opened leaves -> their bodies on the particle list
      if (ptot < 0 || ptot > A.n) {  // more bodies than exist: a corrupt link word
        if (lane == 0) set_status(A.status, BH_ERR_STATE);
        ptot = 0;
      }
      const int pex = pin - np;
      npart += ptot;
      if (!FUSED || bp + ptot <= cap) {
        for (int cb = 0; cb < ptot; cb += 32) {
          const int si = cb + lane;
          int kk = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(kFull, pin, kk + step - 1);
            if (v <= si) kk += step;
          }
          const int of = __shfl_sync(kFull, lk.x, kk);
          const int oe = __shfl_sync(kFull, pex, kk);
          if (si < ptot) {
            const int body = of + (si - oe);
            const int at = bp + si;
            if (at < cap) pl[at] = body;
            psum += (unsigned long long)body;
          }
        }
        bp += ptot;
      } else {  // not enough room: the leaves wait, their bodies are listed as the buffer empties
        const unsigned lb = __ballot_sync(kFull, np > 0);
        __syncwarp();
        if (np > 0) reinterpret_cast<int2 *>(pl + cap)[__popc(lb & lt)] = make_int2(lk.x, np);
        W.npend = __popc(lb);
        W.pend_tot = ptot;
        W.pend_done = 0;
        __syncwarp();
        full = true;  // the caller evaluates the buffers; the next call lists these bodies first
        base += 32;   // this chunk is done (only bodies of its leaves wait)
        break;
      }
    }
    if (full) break;
    __syncwarp();
    int *t = cstk;
    cstk = nstk;
    nstk = t;
    ncur = nnext;
    flip ^= 1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    csum += __shfl_xor_sync(kFull, csum, o);
    psum += __shfl_xor_sync(kFull, psum, o);
  }
  __syncwarp();
  W.depth = depth;
  W.ncur = ncur;
  W.nnext = nnext;
  W.base = base;
  W.flip = flip;
  W.mid = full;
  W.bc = bc;
  W.bp = bp;
  W.ncell = ncell;
  W.npart = npart;
  W.csum = csum;
  W.psum = psum;
  return !full;
}

// The bodies of leaves waiting after pl's cap entries (W.npend leaves, their
// W.pend_tot bodies, W.pend_done of them listed), appended to the particle
// buffer 32 at a time while it has room; W is the walk's state saved in
// memory (lane 0 updates it).  Returns true when all are listed.
__device__ __forceinline__ bool list_waiting(WalkState &W, int *pl, int cap, int lane) {
  const int npend = W.npend, tot = W.pend_tot;
  int pd = W.pend_done, bp = W.bp;
  const int2 pe = (lane < npend) ? reinterpret_cast<const int2 *>(pl + cap)[lane] : make_int2(0, 0);
  int pin = pe.y;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, pin, o);
    if (lane >= o) pin += y;
  }
  const int pex = pin - pe.y;
  unsigned long long psum = 0;
  while (pd < tot && bp + 32 <= cap) {
    const int body = leaf_body(pin, pe.x, pex, pd, tot, lane);
    if (body >= 0) {
      pl[bp + lane] = body;
      psum += (unsigned long long)body;
    }
    const int got = min(32, tot - pd);
    bp += got;
    pd += got;
  }
  for (int o = 16; o > 0; o >>= 1) psum += __shfl_xor_sync(kFull, psum, o);
  __syncwarp();
  if (lane == 0) {
    W.pend_done = pd;
    W.bp = bp;
    W.psum += psum;
  }
  __syncwarp();
  return pd >= tot;
}

// Per-group list statistics and the interaction counters (lane 0).
__device__ __forceinline__ void record_group(const TravArgs &A, int g, int n, const WalkState &W) {
  A.g_npc[g] = W.ncell;
  A.g_npp[g] = W.npart;
  A.g_csum[g] = W.csum;
  A.g_psum[g] = W.psum;
  // every body of the group is on its own particle list once (its own
  // leaves are always opened for theta < 1.15): that self pair is not counted
  const unsigned long long self = (W.npart >= n) ? (unsigned long long)n : 0ull;
  atomicAdd(&A.totals[0], (unsigned long long)n * (unsigned long long)W.npart - self);
  atomicAdd(&A.totals[1], (unsigned long long)n * (unsigned long long)W.ncell);
}

// Split walk, first half: every group's whole lists into one pool at an
// exact offset (one atomic per group), with an estimate of its evaluation
// cost.  A group's pool entry holds its cells, then its bodies.
template <int VAR>
__global__ void __launch_bounds__(kThreads) k_traverse(TravArgs A) {
  const int lane = threadIdx.x & 31;
  WalkState W;
  const size_t gw = (size_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  int *cur = A.stack + gw * 2 * (size_t)A.cap;
  int *nxt = cur + A.cap;
  int *cl = A.scratch + gw * 2 * (size_t)A.list_cap;
  int *pl = cl + A.list_cap;
  const unsigned lt = lanemask_lt();
  const int G = A.counts[1];

  while (true) {
    int g = 0;
    if (lane == 0) g = (int)atomicAdd(A.queue, 1u);
    g = __shfl_sync(kFull, g, 0);
    if (g >= G) break;
    walk_start<VAR>(A, W, g, lane, cur);
    walk_some<VAR, false>(A, W, lane, lt, cur, nxt, cl, pl);
    bool full = false;
    if (W.ncell > A.list_cap || W.npart > A.list_cap) {
      full = true;
      if (lane == 0) set_status(A.status, BH_ERR_CAPACITY);
    }
    // ---- copy the lists into the pool at an exact offset, a multiple of
    // kPoolAlign entries so that offset / kPoolAlign fits the 32-bit field
    const int nc = min(W.ncell, A.list_cap), npp = min(W.npart, A.list_cap);
    unsigned long long off = 0;
    if (lane == 0)
      off = atomicAdd(A.pool_ctr, (unsigned long long)((nc + npp + kPoolAlign - 1) / kPoolAlign * kPoolAlign));
    off = __shfl_sync(kFull, off, 0);
    if (off + (unsigned long long)(nc + npp) > A.pool_cap) {
      full = true;
      if (lane == 0) set_status(A.status, BH_ERR_CAPACITY);
    }
    __syncwarp();
    if (!full) {
      copy_list(A.pool + off, cl, nc, lane);
      copy_list(A.pool + off + nc, pl, npp, lane);
    }
    if (lane == 0) {
      const int n = A.g_beg[g + 1] - A.g_beg[g];
      // evaluation cost ~ (2 cells + 1 body per list entry) / slots per body
      const int P = eval_passes(n);
      const int k = slots_per_body((n + P - 1) / P);
      const int work = full ? 1 : P * ((2 * nc + npp + k - 1) / k + 1);
      A.g_list[g] = full ? make_int4(0, 0, 0, work) : make_int4((int)(unsigned)(off / kPoolAlign), nc, npp, work);
      atomicAdd(&A.work_hist[cost_bucket(work)], 1u);
      record_group(A, g, n, W);
    }
    __syncwarp();
  }
}

// Bucket of a group of n bodies for the fused walk's order (its cost is not
// known before its walk; the body count is the best early estimate).
__device__ __forceinline__ int size_bucket(int n) { return min(max(n, 0), kCostBuckets - 1); }

// Histogram of the group sizes (fused walk); with a flag array, of the
// flagged (active) groups only.
__global__ void __launch_bounds__(256) k_size_hist(const int32_t *__restrict__ counts,
                                                    const int32_t *__restrict__ g_beg,
                                                    const uint8_t *__restrict__ g_active, uint32_t *work_hist) {
  const int G = counts[1];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    if (!g_active || g_active[g]) atomicAdd(&work_hist[size_bucket(g_beg[g + 1] - g_beg[g])], 1u);
}

// Places the groups in order of decreasing estimated cost: the groups of
// bucket b take the slots after those of every costlier bucket (in any order
// within the bucket; a group's result does not depend on when it is taken).
// Every block recomputes the bucket offsets from the histogram; appends are
// aggregated per warp over lanes of equal bucket.
template <bool BY_SIZE>
__global__ void __launch_bounds__(kCostBuckets) k_order(int32_t *counts, const int4 *__restrict__ g_list,
                                                         const int32_t *__restrict__ g_beg,
                                                         const uint8_t *__restrict__ g_active, uint32_t *work_hist,
                                                         int32_t *order) {
  __shared__ uint32_t s_start[kCostBuckets];
  __shared__ uint32_t s_warp[kCostBuckets / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  // exclusive prefix over the buckets from the costliest down: thread t holds bucket 255 - t
  const uint32_t v = work_hist[kCostBuckets - 1 - t];
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  uint32_t off = 0;
  for (int i = 0; i < w; ++i) off += s_warp[i];
  s_start[kCostBuckets - 1 - t] = off + x - v;
  if (blockIdx.x == 0 && t == kCostBuckets - 1) counts[3] = (int32_t)(off + x);  // groups placed: the walk's count
  __syncthreads();
  const int G = counts[1];
  uint32_t *fill = work_hist + kCostBuckets;
  const unsigned lt = lanemask_lt();
  for (int base = blockIdx.x * blockDim.x; base < G; base += gridDim.x * blockDim.x) {
    const int g = base + t;
    const int b = (g >= G || (g_active && !g_active[g])) ? -1
                  : BY_SIZE ? size_bucket(g_beg[g + 1] - g_beg[g]) : cost_bucket(g_list[g].w);
    const unsigned peers = __match_any_sync(kFull, b);
    const int leader = __ffs(peers) - 1;
    uint32_t first = 0;
    if (lane == leader && b >= 0) first = atomicAdd(&fill[b], (uint32_t)__popc(peers));
    first = __shfl_sync(kFull, first, leader);
    if (b >= 0) {
      const uint32_t pos = s_start[b] + first + (uint32_t)__popc(peers & lt);
      if (pos < (uint32_t)G) order[pos] = g;
    }
  }
}

// =============================================================== evaluation
struct EvalSmem {
  // staged cells: (dx, dy, dz, M), -(Qxx, Qyy, Qzz, Qxy), -(Qxz, Qyz, 0, 0)
  float4 sc[kStage][3];
  // staged bodies: (S_hi, m), (S_lo, 0) -- the rounded offset and its residual
  float4 sp[kStage][2];
  int pidx[kStage];  // their sorted indices (read only for tiles holding the group's own bodies)
  float4 ah[64];     // per slot: compensated sum (hi part) of acceleration and potential
  float4 al[64];     // per slot: its lo part
};

struct EvalArgs {
  const float4 *__restrict__ part_hi;
  const float4 *__restrict__ part_lo;
  const float4 *__restrict__ mom;
  const int32_t *__restrict__ g_beg;
  const int4 *__restrict__ g_list;
  const uint32_t *__restrict__ pool;
  const int32_t *__restrict__ counts;  // [1] groups, [3] groups in the order
  const int32_t *__restrict__ order;  // groups, most expensive first
  float eps2;
  uint32_t *queue;
  float4 *acc_sorted;
  float *acc_out;
  float *pot_out;
  const uint32_t *__restrict__ perm;
  float4 *hold;  // [2 N] per body (sorted order): (hi, lo) sums between parts of a list (fused walk)
};

// The two target slots of a lane, as pairs (slot 0 in .x, slot 1 in .y).  The
// offsets are kept negated so that a difference is one packed add.
struct Targets2 {
  float2 nhx, nhy, nhz;  // -(rounded offset from the group centre)
  float2 nlx, nly, nlz;  // -(its residual)
};

// Partial sums of a lane's two slots since the last fold; the potential is
// accumulated with the opposite sign (-phi).
struct Acc2 {
  float2 x, y, z, np;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Fold a slot's partial sum into its compensated (hi, lo) pair, which lives in
// shared memory (touched once per ~64 interactions, so not worth registers).
template <int VAR>
__device__ __forceinline__ void fold(float4 &hs, float4 &ls, float x, float y, float z, float p) {
  float4 hi = hs, lo = ls;
  if (relative(VAR)) {
    two_sum_into(hi.x, lo.x, x);
    two_sum_into(hi.y, lo.y, y);
    two_sum_into(hi.z, lo.z, z);
    two_sum_into(hi.w, lo.w, p);
    ls = lo;
  } else {
    hi.x += x;
    hi.y += y;
    hi.z += z;
    hi.w += p;
  }
  hs = hi;
}

template <int VAR>
__device__ __forceinline__ void fold2(EvalSmem &S, int lane, Acc2 &t) {
  fold<VAR>(S.ah[lane], S.al[lane], t.x.x, t.y.x, t.z.x, -t.np.x);
  fold<VAR>(S.ah[32 + lane], S.al[32 + lane], t.x.y, t.y.y, t.z.y, -t.np.y);
  const float2 z = f2(0.f, 0.f);
  t = Acc2{z, z, z, z};
}

// Softened particle-particle interaction of one staged source with both slots
// of a lane, in packed FP32 pairs: 20 flops per slot by the convention FMA = 2,
// rsqrt = 1 (the two-float difference d = (S_hi - T_hi) + (S_lo - T_lo) costs 6
// more: its first term is exact for close pairs, so a pair keeps its relative
// accuracy however far it is from the group centre).  SELF: skip the pair of a
// body with itself (same index); GUARD: eps = 0, zero distances skipped.
template <int VAR, bool GUARD, bool SELF>
__device__ __forceinline__ void pp2(Acc2 &a, const Targets2 &t, const float4 sh, const float4 sl, float2 e2,
                                    int me0 = 0, int me1 = 0, int other = -1) {
  float2 dx, dy, dz;
  if (relative(VAR)) {
    dx = __fadd2_rn(__fadd2_rn(f2(sh.x, sh.x), t.nhx), __fadd2_rn(f2(sl.x, sl.x), t.nlx));
    dy = __fadd2_rn(__fadd2_rn(f2(sh.y, sh.y), t.nhy), __fadd2_rn(f2(sl.y, sl.y), t.nly));
    dz = __fadd2_rn(__fadd2_rn(f2(sh.z, sh.z), t.nhz), __fadd2_rn(f2(sl.z, sl.z), t.nlz));
  } else {
    dx = __fadd2_rn(f2(sh.x, sh.x), t.nhx);
    dy = __fadd2_rn(f2(sh.y, sh.y), t.nhy);
    dz = __fadd2_rn(f2(sh.z, sh.z), t.nhz);
  }
  float2 r2 = __ffma2_rn(dx, dx, e2);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dz, dz, r2);
  float2 ri = f2(rsqrtf(r2.x), rsqrtf(r2.y));
  if (GUARD) {
    ri.x = (r2.x > 0.f) ? ri.x : 0.f;
    ri.y = (r2.y > 0.f) ? ri.y : 0.f;
  }
  if (SELF) {
    ri.x = (me0 == other) ? 0.f : ri.x;
    ri.y = (me1 == other) ? 0.f : ri.y;
  }
  const float2 mr = __fmul2_rn(f2(sh.w, sh.w), ri);
  const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
  a.np = __fadd2_rn(a.np, mr);
  a.x = __ffma2_rn(mr3, dx, a.x);
  a.y = __ffma2_rn(mr3, dy, a.y);
  a.z = __ffma2_rn(mr3, dz, a.z);
}

// Softened particle-cell interaction, monopole + quadrupole, of one staged cell
// with both slots of a lane, with d = com - target:
//   a = M d/s^3 - Q d/s^5 + (5/2)(d.Q.d) d/s^7,  phi = -M/s - (d.Q.d)/(2 s^5),
// rearranged as a = (q + s^2 (M - (5/2) w/s^4) d)/s^5 with q = -Q d and
// w = -d.Q.d (the staged Q is negated, so both come out of plain products):
// 32 packed operations per slot pair, 53 flops per slot by the counting rule
// (the work unit stays the 54 flops fixed from the first sequence).
__device__ __forceinline__ void pc2(Acc2 &a, const Targets2 &t, const float4 c0, const float4 q0, const float4 q1,
                                    float2 e2) {
  const float2 dx = __fadd2_rn(f2(c0.x, c0.x), t.nhx);
  const float2 dy = __fadd2_rn(f2(c0.y, c0.y), t.nhy);
  const float2 dz = __fadd2_rn(f2(c0.z, c0.z), t.nhz);
  float2 r2 = __ffma2_rn(dx, dx, e2);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dz, dz, r2);
  const float2 ri = f2(rsqrtf(r2.x), rsqrtf(r2.y));
  const float2 ri2 = __fmul2_rn(ri, ri);
  const float2 M = f2(c0.w, c0.w);
  const float2 qxx = f2(q0.x, q0.x), qyy = f2(q0.y, q0.y), qzz = f2(q0.z, q0.z);
  const float2 qxy = f2(q0.w, q0.w), qxz = f2(q1.x, q1.x), qyz = f2(q1.y, q1.y);
  const float2 qx = __ffma2_rn(qxz, dz, __ffma2_rn(qxy, dy, __fmul2_rn(qxx, dx)));
  const float2 qy = __ffma2_rn(qyz, dz, __ffma2_rn(qyy, dy, __fmul2_rn(qxy, dx)));
  const float2 qz = __ffma2_rn(qzz, dz, __ffma2_rn(qyz, dy, __fmul2_rn(qxz, dx)));
  const float2 w = __ffma2_rn(qz, dz, __ffma2_rn(qy, dy, __fmul2_rn(qx, dx)));
  const float2 ri4 = __fmul2_rn(ri2, ri2);
  const float2 ri5 = __fmul2_rn(ri4, ri);
  const float2 u = __fmul2_rn(w, ri4);  // w / s^4
  // a = (q + c d) / s^5 with c = s^2 (M - (5/2) u);  -phi += (M - u / 2) / s
  const float2 c = __fmul2_rn(r2, __ffma2_rn(f2(-2.5f, -2.5f), u, M));
  a.np = __ffma2_rn(__ffma2_rn(f2(-0.5f, -0.5f), u, M), ri, a.np);
  a.x = __ffma2_rn(ri5, __ffma2_rn(c, dx, qx), a.x);
  a.y = __ffma2_rn(ri5, __ffma2_rn(c, dy, qy), a.y);
  a.z = __ffma2_rn(ri5, __ffma2_rn(c, dz, qz), a.z);
}

// Shared-memory staging: entries kTile..kStage-1 are permanent nulls (zero mass, far away).
__device__ __forceinline__ void init_stage(EvalSmem &S, int lane) {
  const float4 null_src = make_float4(kFar, kFar, kFar, 0.f);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (lane < kStage - kTile) {
    S.sc[kTile + lane][0] = null_src;
    S.sc[kTile + lane][1] = zero4;
    S.sc[kTile + lane][2] = zero4;
    S.sp[kTile + lane][0] = null_src;
    S.sp[kTile + lane][1] = zero4;
    S.pidx[kTile + lane] = -1;
  }
  __syncwarp();
}

// Accelerations and potentials of group g's bodies from (a part of) its cell
// list clist[0..nc) and particle list plist[0..np), by one warp.
//
// The lists may come in parts (the fused walk evaluates its buffers whenever
// they fill): `first` starts every body's sums at zero, `last` writes the
// results.  Between parts a one-pass group keeps its slots' compensated sums
// in shared memory; a group of several passes keeps, per body, the slots'
// sums combined into one (hi, lo) pair in A.hold (sorted body order), and
// restores it into the body's first slot.
template <int VAR, bool GUARD, int MODE>
__device__ __forceinline__ void eval_lists(const EvalArgs &A, EvalSmem &S, int lane, int g, const uint32_t *clist,
                                           int nc, const uint32_t *plist, int np, bool first, bool last) {
  const float2 e2 = f2(A.eps2, A.eps2);
  const float4 null_src = make_float4(kFar, kFar, kFar, 0.f);  // far away, zero mass, no quadrupole
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const int gb0 = A.g_beg[g];
  const int ng = A.g_beg[g + 1] - gb0;
  float cx = 0.f, cy = 0.f, cz = 0.f;
  if (relative(VAR)) {
    const float4 c = A.part_hi[gb0];
    cx = c.x;
    cy = c.y;
    cz = c.z;
  }
  const int npass = eval_passes(ng);
  const int nbp = (ng + npass - 1) / npass;
  for (int pass = 0; pass < npass; ++pass) {
    // this pass: bodies gb .. gb + n - 1 of the group, on the group's lists
    const int gb = gb0 + pass * nbp;
    const int n = min(nbp, ng - pass * nbp);
    // lane -> (phase ph, bodies b0 and b1 = b0 + h): both slots read the same entry
    const int h = pair_stride(n);
    const int k = 32 / h;  // phases = slots per body
    const int ph = min(lane / h, k - 1);
    const int b0 = lane % h, b1 = b0 + h;
    const bool v0 = lane < h * k && b0 < n, v1 = lane < h * k && b1 < n;
    // body b's first slot: b (k = 1: b < 32) or 32 + b - 32 (k = 1: b >= 32);
    // for k > 1, b for b < h and 32 + b - h otherwise
    const int s0 = (lane < h) ? lane : 32 + lane - h;
    Targets2 T;
    {
      const int lb0 = gb + min(b0, n - 1), lb1 = gb + min(b1, n - 1);
      const Target t0 = make_target<VAR>(A.part_hi[lb0], A.part_lo[lb0], cx, cy, cz);
      const Target t1 = make_target<VAR>(A.part_hi[lb1], A.part_lo[lb1], cx, cy, cz);
      T.nhx = f2(-t0.hx, -t1.hx);
      T.nhy = f2(-t0.hy, -t1.hy);
      T.nhz = f2(-t0.hz, -t1.hz);
      T.nlx = f2(-t0.lx, -t1.lx);
      T.nly = f2(-t0.ly, -t1.ly);
      T.nlz = f2(-t0.lz, -t1.lz);
    }
    if (first || npass > 1) {
      S.ah[lane] = zero4;
      S.al[lane] = zero4;
      S.ah[32 + lane] = zero4;
      S.al[32 + lane] = zero4;
      if (!first) {  // several passes: this pass's sums so far, one pair per body, into its first slot
        __syncwarp();
        if (k == 1) {
          if (v0) {
            S.ah[lane] = A.hold[2 * (gb + b0)];
            S.al[lane] = A.hold[2 * (gb + b0) + 1];
          }
          if (v1) {
            S.ah[32 + lane] = A.hold[2 * (gb + b1)];
            S.al[32 + lane] = A.hold[2 * (gb + b1) + 1];
          }
        } else if (lane < n) {
          S.ah[s0] = A.hold[2 * (gb + lane)];
          S.al[s0] = A.hold[2 * (gb + lane) + 1];
        }
      }
    }
    Acc2 t;  // partial sums since the last fold
    t.x = t.y = t.z = t.np = f2(0.f, 0.f);
    int since = 0;  // interactions per slot since the last fold

    // ---- cell list, kTile entries at a time (each lane stages two)
    {
      for (int base = 0; base < nc; base += kTile) {
        const int cnt = min(kTile, nc - base);
#pragma unroll
        for (int hh = 0; hh < kTile / 32; ++hh) {
          const int e = hh * 32 + lane;
          if (e < cnt) {
            const size_t ci = clist[base + e];
            const float4 ra = A.mom[4 * ci], rb = A.mom[4 * ci + 1], rq0 = A.mom[4 * ci + 2],
                         rq1 = A.mom[4 * ci + 3];
            float dx, dy, dz;
            if (relative(VAR)) {
              dx = (ra.x - cx) + rb.x;
              dy = (ra.y - cy) + rb.y;
              dz = (ra.z - cz) + rb.z;
            } else {
              dx = ra.x;
              dy = ra.y;
              dz = ra.z;
            }
            S.sc[e][0] = make_float4(dx, dy, dz, ra.w);
            S.sc[e][1] = make_float4(-rq0.x, -rq0.y, -rq0.z, -rq0.w);
            S.sc[e][2] = make_float4(-rq1.x, -rq1.y, 0.f, 0.f);
          } else {
            S.sc[e][0] = null_src;
            S.sc[e][1] = zero4;
            S.sc[e][2] = zero4;
          }
        }
        __syncwarp();
#pragma unroll 1
        for (int j = ph; j < cnt + ph; j += k) {
          const float4 *e = S.sc[j];
          pc2(t, T, e[0], e[1], e[2], e2);
        }
        since += (cnt + k - 1) / k;
        if (since >= kFoldEvery) {
          fold2<VAR>(S, lane, t);
          since = 0;
        }
        __syncwarp();
      }
    }
    // ---- particle list, kTile entries at a time (each lane stages two)
    {
      for (int base = 0; base < np; base += kTile) {
        const int cnt = min(kTile, np - base);
        bool member = false;
#pragma unroll
        for (int hh = 0; hh < kTile / 32; ++hh) {
          const int e = hh * 32 + lane;
          if (e < cnt) {
            const int rb = (int)plist[base + e];
            const float4 rh = A.part_hi[rb], rl = A.part_lo[rb];
            member |= (unsigned)(rb - gb) < (unsigned)n;
            const Target s = make_target<VAR>(rh, rl, cx, cy, cz);
            S.sp[e][0] = make_float4(s.hx, s.hy, s.hz, rh.w);
            S.sp[e][1] = make_float4(s.lx, s.ly, s.lz, 0.f);
            S.pidx[e] = rb;
          } else {
            S.sp[e][0] = null_src;
            S.sp[e][1] = zero4;
            S.pidx[e] = -1;
          }
        }
        const bool self_tile = __any_sync(kFull, member);
        __syncwarp();
        if (self_tile) {
          // a tile with the group's own bodies: skip each body's pair with itself by index
          const int me0 = gb + b0, me1 = gb + b1;
          for (int j = ph; j < cnt + ph; j += k) {
            const float4 *e = S.sp[j];
            pp2<VAR, GUARD, true>(t, T, e[0], e[1], e2, me0, me1, S.pidx[j]);
          }
        } else {
#pragma unroll 2
          for (int j = ph; j < cnt + ph; j += k) {
            const float4 *e = S.sp[j];
            pp2<VAR, GUARD, false>(t, T, e[0], e[1], e2);
          }
        }
        since += (cnt + k - 1) / k;
        if (since >= kFoldEvery) {
          fold2<VAR>(S, lane, t);
          since = 0;
        }
        __syncwarp();
      }
    }
    fold2<VAR>(S, lane, t);
    __syncwarp();

    // ---- combine the slots of each body: write the results, or (several
    // passes, more parts to come) keep the pair
    auto put_body = [&](int b, const float4 &H, const float4 &Lo) {
      const int gi = gb + b;
      if (!last) {
        A.hold[2 * gi] = H;
        A.hold[2 * gi + 1] = Lo;
      } else if (MODE == kOutSorted) {
        A.acc_sorted[gi] = make_float4(H.x + Lo.x, H.y + Lo.y, H.z + Lo.z, H.w + Lo.w);
      } else {
        const size_t j = A.perm[gi];
        A.acc_out[3 * j] = H.x + Lo.x;
        A.acc_out[3 * j + 1] = H.y + Lo.y;
        A.acc_out[3 * j + 2] = H.z + Lo.z;
        A.pot_out[j] = H.w + Lo.w;
      }
    };
    if (last || npass > 1) {
      if (k == 1) {
        if (v0) put_body(b0, S.ah[lane], S.al[lane]);
        if (v1) put_body(b1, S.ah[32 + lane], S.al[32 + lane]);
      } else if (lane < n) {
        // body b's slots: b + q h (q < k) in the first half of the slot array
        // for b < h, b - h + q h in the second half otherwise
        float4 H = S.ah[s0], Lo = S.al[s0];
        for (int q = 1; q < k; ++q) {
          const float4 hq = S.ah[s0 + q * h], lq = S.al[s0 + q * h];
          two_sum_into(H.x, Lo.x, hq.x);
          two_sum_into(H.y, Lo.y, hq.y);
          two_sum_into(H.z, Lo.z, hq.z);
          two_sum_into(H.w, Lo.w, hq.w);
          Lo.x += lq.x;
          Lo.y += lq.y;
          Lo.z += lq.z;
          Lo.w += lq.w;
        }
        put_body(lane, H, Lo);
      }
    }
    __syncwarp();
  }  // passes
}

// Split walk, second half: every group's lists from the pool, most expensive
// group first, so that the launch ends on cheap ones.
template <int VAR, bool GUARD, int MODE>
__global__ void __launch_bounds__(kThreads, kEvalMinBlocks) k_eval(EvalArgs A) {
  extern __shared__ EvalSmem s_eval[];
  const int lane = threadIdx.x & 31;
  EvalSmem &S = s_eval[threadIdx.x >> 5];
  init_stage(S, lane);
  const int G = A.counts[1], NQ = A.counts[3];  // groups; groups in the order
  while (true) {
    int q = 0;
    if (lane == 0) q = (int)atomicAdd(A.queue, 1u);
    q = __shfl_sync(kFull, q, 0);
    if (q >= NQ) break;
    const int g = A.order[q];
    if ((unsigned)g >= (unsigned)G) continue;  // (never: k_order fills every slot)
    const int4 L = A.g_list[g];  // {offset / kPoolAlign, cells, bodies, cost}: cells, then bodies
    const uint32_t *lst = A.pool + (size_t)kPoolAlign * (unsigned)L.x;
    // pull the group's lists from DRAM into L2 now (one 128-byte line per 32 entries)
    for (int i = 32 * lane; i < L.y + L.z; i += 32 * 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(lst + i));
    eval_lists<VAR, GUARD, MODE>(A, S, lane, g, lst, L.y, lst + L.y, L.z, true, true);
  }
}

// Fused walk: a warp alternates between walking its group (walk_some, the
// walk's state kept in shared memory) and evaluating the group's list
// buffers: whenever a buffer of list_buffer entries fills, the whole tiles
// of both buffers are evaluated and the rest moves to their fronts; when the
// walk ends, everything left (§2.2, Fig. 3: lists are evaluated as they
// fill, the remainder at the end).  The buffers (per warp: list_buffer cells
// and as many bodies) stay in L2, and no list length is limited.  Walk and
// evaluation are each inlined once, so each has the kernel's registers to
// itself.  Groups are taken largest first; one warp's walk overlaps other
// warps' evaluations on the SM (the walk is issue- and latency-bound on the
// integer and load pipes, the evaluation bound by the FP32 pipe).
template <int VAR, bool GUARD, int MODE>
__global__ void __launch_bounds__(kThreads, kWalkMinBlocks) k_walk(TravArgs T, EvalArgs E) {
  extern __shared__ EvalSmem s_eval[];
  const int lane = threadIdx.x & 31;
  EvalSmem &S = s_eval[threadIdx.x >> 5];
  init_stage(S, lane);
  // this warp's stacks and buffers (recomputed where used: fewer live registers)
  auto gw = [&]() { return (size_t)blockIdx.x * kWarps + (threadIdx.x >> 5); };
  auto stk = [&]() { return T.stack + gw() * 2 * (size_t)T.cap; };
  auto cls = [&]() { return T.scratch + gw() * (size_t)walk_stride(T.list_cap); };  // cells, bodies, waiting leaves
  auto saved = [&]() -> WalkState & {
    return *reinterpret_cast<WalkState *>(cls() + 2 * (size_t)T.list_cap + 64);
  };
  const int G = T.counts[1], NQ = T.counts[3];  // groups; groups in the order (the active ones)
  while (true) {
    int q = 0;
    if (lane == 0) q = (int)atomicAdd(E.queue, 1u);
    q = __shfl_sync(kFull, q, 0);
    if (q >= NQ) break;
    const int g = E.order[q];
    if ((unsigned)g >= (unsigned)G) continue;  // (never: k_order fills every slot)
    WalkState W;  // the walk's state, in registers while the warp walks
    walk_start<VAR>(T, W, g, lane, stk());
    for (int parts = 0;; ++parts) {
      const bool done = walk_some<VAR, true>(T, W, lane, lanemask_lt(), stk(), stk() + T.cap, cls(),
                                             cls() + T.list_cap);
      int wc = W.bc, wp = W.bp;  // everything at the walk's end
      if (done) {
        if (lane == 0) record_group(T, g, T.g_beg[g + 1] - T.g_beg[g], W);
      } else {  // whole tiles now; the state waits in the scratch meanwhile
        wc &= ~(kTile - 1);
        wp &= ~(kTile - 1);
        if (lane == 0) saved() = W;
      }
      __syncwarp();
      const uint32_t *c = reinterpret_cast<const uint32_t *>(cls());
      if (parts == 0 && done)  // the common case: the whole lists in one evaluation
        eval_lists<VAR, GUARD, MODE>(E, S, lane, g, c, wc, c + T.list_cap, wp, true, true);
      else
        eval_lists<VAR, GUARD, MODE>(E, S, lane, g, c, wc, c + T.list_cap, wp, parts == 0, done);
      if (done) break;
      // the rest of each buffer (fewer than kTile entries) to its front, then
      // the bodies of waiting leaves, evaluating the particle buffer whenever
      // it fills
      WalkState &M = saved();
      int *cl = cls(), *pl = cl + T.list_cap;
      while (true) {
        const int bc = M.bc, bp = M.bp;
        const int mc = bc & ~(kTile - 1), mp = bp & ~(kTile - 1);
        const int rc = bc - mc, rp = bp - mp;
        int c0 = 0, c1 = 0, p0 = 0, p1 = 0;
        if (lane < rc) c0 = cl[mc + lane];
        if (32 + lane < rc) c1 = cl[mc + 32 + lane];
        if (lane < rp) p0 = pl[mp + lane];
        if (32 + lane < rp) p1 = pl[mp + 32 + lane];
        __syncwarp();
        if (lane < rc) cl[lane] = c0;
        if (32 + lane < rc) cl[32 + lane] = c1;
        if (lane < rp) pl[lane] = p0;
        if (32 + lane < rp) pl[32 + lane] = p1;
        if (lane == 0) {
          M.bc = rc;
          M.bp = rp;
        }
        __syncwarp();
        if (M.pend_done >= M.pend_tot || list_waiting(M, pl, T.list_cap, lane)) break;
        ++parts;  // the particle buffer is full again: its whole tiles
        eval_lists<VAR, GUARD, MODE>(E, S, lane, g, c, 0, c + T.list_cap, M.bp & ~(kTile - 1), false, false);
      }
      W = M;
    }
  }
}

// FP64 evaluation of the same lists (walk variant 2, a precision reference on
// the GPU: GB300's FP64 rate is a small fraction of its FP32 rate, so this is a
// study variant, not a fast path).  One warp per group, a lane per body (two
// for n > 32), positions recombined from their two-float form (~2^-48 relative),
// moments as stored (FP32), every operation in FP64.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_eval_f64(EvalArgs A) {
  const int lane = threadIdx.x & 31;
  const double eps2 = (double)A.eps2;
  const int G = A.counts[1];
  while (true) {
    int g = 0;
    if (lane == 0) g = (int)atomicAdd(A.queue, 1u);
    g = __shfl_sync(kFull, g, 0);
    if (g >= G) break;
    const int gb = A.g_beg[g];
    const int n = A.g_beg[g + 1] - gb;
    const int4 L = A.g_list[g];  // cells, then bodies
    const uint32_t *clist = A.pool + (size_t)kPoolAlign * (unsigned)L.x;
    const uint32_t *plist = clist + L.y;
    for (int b = lane; b < n; b += 32) {  // (one sweep: this study variant is not tuned)
      const float4 th = A.part_hi[gb + b], tl = A.part_lo[gb + b];
      const double tx = (double)th.x + (double)tl.x, ty = (double)th.y + (double)tl.y,
                   tz = (double)th.z + (double)tl.z;
      double ax = 0, ay = 0, az = 0, ap = 0;
      for (int j = 0; j < L.y; ++j) {
        const size_t c = clist[j];
        const float4 a = A.mom[4 * c], lo = A.mom[4 * c + 1], q0 = A.mom[4 * c + 2], q1 = A.mom[4 * c + 3];
        const double dx = ((double)a.x + (double)lo.x) - tx, dy = ((double)a.y + (double)lo.y) - ty,
                     dz = ((double)a.z + (double)lo.z) - tz;
        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
        const double ri = 1.0 / sqrt(r2), ri2 = ri * ri, ri5 = ri2 * ri2 * ri;
        const double qx = (double)q0.x * dx + (double)q0.w * dy + (double)q1.x * dz;
        const double qy = (double)q0.w * dx + (double)q0.y * dy + (double)q1.y * dz;
        const double qz = (double)q1.x * dx + (double)q1.y * dy + (double)q0.z * dz;
        const double dqd = qx * dx + qy * dy + qz * dz;
        const double mr = (double)a.w * ri;
        const double coef = mr * ri2 + 2.5 * dqd * ri5 * ri2;
        ax += coef * dx - ri5 * qx;
        ay += coef * dy - ri5 * qy;
        az += coef * dz - ri5 * qz;
        ap += -mr - 0.5 * dqd * ri5;
      }
      for (int j = 0; j < L.z; ++j) {
        const int s = (int)plist[j];
        if (s == gb + b) continue;
        const float4 sh = A.part_hi[s], sl = A.part_lo[s];
        const double dx = ((double)sh.x + (double)sl.x) - tx, dy = ((double)sh.y + (double)sl.y) - ty,
                     dz = ((double)sh.z + (double)sl.z) - tz;
        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
        if (!(r2 > 0.0)) continue;
        const double ri = 1.0 / sqrt(r2);
        const double mr = (double)sh.w * ri, mr3 = mr * ri * ri;
        ax += mr3 * dx;
        ay += mr3 * dy;
        az += mr3 * dz;
        ap -= mr;
      }
      const int gi = gb + b;
      if (MODE == kOutSorted) {
        A.acc_sorted[gi] = make_float4((float)ax, (float)ay, (float)az, (float)ap);
      } else {
        const size_t o = A.perm[gi];
        A.acc_out[3 * o] = (float)ax;
        A.acc_out[3 * o + 1] = (float)ay;
        A.acc_out[3 * o + 2] = (float)az;
        A.pot_out[o] = (float)ap;
      }
    }
  }
}

template <int VAR, bool GUARD, int MODE>
cudaError_t launch_eval(Ctx &c, const EvalArgs &a, cudaStream_t s) {
  k_eval<VAR, GUARD, MODE><<<c.eval_grid, kThreads, kWarps * sizeof(EvalSmem), s>>>(a);
  return cudaGetLastError();
}

template <int VAR, bool GUARD, int MODE>
cudaError_t launch_fused(Ctx &c, const TravArgs &t, const EvalArgs &a, cudaStream_t s) {
  k_walk<VAR, GUARD, MODE><<<c.walk_grid, kThreads, kWarps * sizeof(EvalSmem), s>>>(t, a);
  return cudaGetLastError();
}

}  // namespace

namespace {
// g_active[g] = 1 for groups g0 <= g < g1 of the last build, else 0.
__global__ void __launch_bounds__(256) k_mark_groups(const int32_t *__restrict__ counts, int g0, int g1,
                                                     uint8_t *g_active) {
  const int G = counts[1];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
    g_active[g] = (g >= g0 && g < g1) ? 1 : 0;
}
}  // namespace

cudaError_t launch_mark_groups(Ctx &c, int g0, int g1, cudaStream_t s) {
  k_mark_groups<<<c.num_sms * 4, 256, 0, s>>>(c.d_counts, g0, g1, c.g_active);
  c.launches++;
  return cudaGetLastError();
}

int walk_smem_bytes(int warps) { return warps * (int)sizeof(EvalSmem); }

// Ints of list scratch per walking warp: the fused walk's buffers, or for
// the split walk two lists of list_capacity entries (or the buffers if
// larger: a walk restricted to active groups is always fused).
int walk_list_stride(const bh_params &p) {
  const long fused = walk_stride(p.list_buffer), split = 2L * p.list_capacity;
  return (int)((walk_is_fused(p) || fused > split) ? fused : split);
}

cudaError_t walk_init_attrs(int smem) {
  cudaError_t e = cudaSuccess;
#define BH_EVAL_ATTR(V, G, M)                                                                        \
  if (!e) e = cudaFuncSetAttribute(k_eval<V, G, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
  if (!e) e = cudaFuncSetAttribute(k_walk<V, G, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  BH_EVAL_ATTR(0, false, kOutCaller)
  BH_EVAL_ATTR(0, true, kOutCaller)
  BH_EVAL_ATTR(0, false, kOutSorted)
  BH_EVAL_ATTR(0, true, kOutSorted)
  BH_EVAL_ATTR(1, false, kOutCaller)
  BH_EVAL_ATTR(1, true, kOutCaller)
  BH_EVAL_ATTR(1, false, kOutSorted)
  BH_EVAL_ATTR(1, true, kOutSorted)
  BH_EVAL_ATTR(kVarDeep, false, kOutCaller)
  BH_EVAL_ATTR(kVarDeep, true, kOutCaller)
  BH_EVAL_ATTR(kVarDeep, false, kOutSorted)
  BH_EVAL_ATTR(kVarDeep, true, kOutSorted)
#undef BH_EVAL_ATTR
  return e;
}

void walk_grids(int *trav_blocks_per_sm, int *eval_blocks_per_sm, int *fused_blocks_per_sm) {
  int nt = 0, ne = 0, nf = 0;
  const int smem = kWarps * (int)sizeof(EvalSmem);
  cudaFuncSetAttribute(k_eval<0, false, kOutCaller>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_walk<0, false, kOutCaller>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nt, k_traverse<0>, kThreads, 0) != cudaSuccess) nt = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ne, k_eval<0, false, kOutCaller>, kThreads, smem) !=
      cudaSuccess)
    ne = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nf, k_walk<0, false, kOutCaller>, kThreads, smem) !=
      cudaSuccess)
    nf = 1;
  *trav_blocks_per_sm = nt > 0 ? nt : 1;
  *eval_blocks_per_sm = ne > 0 ? ne : 1;
  *fused_blocks_per_sm = nf > 0 ? nf : 1;
}

int walk_block_warps() { return kWarps; }

cudaError_t launch_walk(Ctx &c, float theta, float eps, OutMode mode, float *acc, float *pot, cudaStream_t s,
                        const uint8_t *g_active) {
  TravArgs t;
  t.part_hi = c.part_hi;
  t.part_lo = c.part_lo;
  t.mac = c.c_mac;
  t.mac_lo = c.c_mac_lo;
  t.link = c.c_link;
  t.g_beg = c.g_beg;
  t.g_sys = c.g_sys;
  t.sys_root = c.sys_root;
  t.counts = c.d_counts;
  t.stack = c.walk_stack;
  t.cap = c.p.stack_capacity;
  t.scratch = c.list_scratch;
  // the fused walk's bounded buffers, or the split walk's whole lists
  t.list_cap = (walk_is_fused(c.p) || g_active) ? c.p.list_buffer : c.p.list_capacity;
  t.pool = c.list_pool;
  t.pool_cap = (unsigned long long)c.pool_cap;
  t.pool_ctr = c.pool_ctr;
  t.g_list = c.g_list;
  t.work_hist = c.work_hist;
  t.box_mac = c.p.mac;
  t.two_over_theta = (theta > 0.f) ? 2.0f / theta : INFINITY;
  t.n = (int)c.n;
  t.queue = c.walk_queue;
  t.g_npc = c.g_npc;
  t.g_npp = c.g_npp;
  t.g_csum = c.g_csum;
  t.g_psum = c.g_psum;
  t.totals = c.d_totals;
  t.status = c.d_status;
  EvalArgs a;
  a.part_hi = c.part_hi;
  a.part_lo = c.part_lo;
  a.mom = c.c_mom;
  a.g_beg = c.g_beg;
  a.g_list = c.g_list;
  a.pool = c.list_pool;
  a.counts = c.d_counts;
  a.order = c.g_order;
  a.eps2 = eps * eps;
  a.queue = c.walk_queue + 1;
  a.acc_sorted = c.acc_sorted;
  a.acc_out = acc;
  a.pot_out = pot;
  a.perm = c.idx[0];
  a.hold = c.acc_hold;
  // keys deeper than 20 levels take the deep form of variant 0 (and of the FP64 variant's walk)
  const bool deep = c.levels > kLevels;
  const int var = (c.p.walk_variant == 0 && deep) ? kVarDeep : c.p.walk_variant;
  const bool guard = !(a.eps2 > 0.f);
  const bool fused = walk_is_fused(c.p) || g_active;  // a walk of some groups only is always fused
  cudaError_t e = cudaSuccess;
  auto mark = [&](int end) {
    if (!c.profiling) return;
    if (c.capturing) cudaEventRecordWithFlags(c.ev[8][end], s, cudaEventRecordExternal);
    else cudaEventRecord(c.ev[8][end], s);
    if (end) c.phase_rec[8] = true;
  };
  if (fused) {
    // groups by size (largest first), then one kernel walks and evaluates
    k_size_hist<<<c.num_sms * 4, 256, 0, s>>>(c.d_counts, c.g_beg, g_active, c.work_hist);
    e = cudaGetLastError();
    c.launches++;
    if (e) return e;
    k_order<true><<<c.num_sms * 4, kCostBuckets, 0, s>>>(c.d_counts, c.g_list, c.g_beg, g_active, c.work_hist,
                                                         c.g_order);
    e = cudaGetLastError();
    c.launches++;
    if (e) return e;
    mark(0);
#define BH_WALK_CASE(V, G, M) \
  if (var == V && guard == G && mode == M) e = launch_fused<V, G, M>(c, t, a, s); else
    BH_WALK_CASE(0, false, kOutCaller)
    BH_WALK_CASE(0, true, kOutCaller)
    BH_WALK_CASE(0, false, kOutSorted)
    BH_WALK_CASE(0, true, kOutSorted)
    BH_WALK_CASE(1, false, kOutCaller)
    BH_WALK_CASE(1, true, kOutCaller)
    BH_WALK_CASE(1, false, kOutSorted)
    BH_WALK_CASE(1, true, kOutSorted)
    BH_WALK_CASE(kVarDeep, false, kOutCaller)
    BH_WALK_CASE(kVarDeep, true, kOutCaller)
    BH_WALK_CASE(kVarDeep, false, kOutSorted)
    BH_WALK_CASE(kVarDeep, true, kOutSorted)
    e = cudaErrorInvalidValue;
#undef BH_WALK_CASE
    mark(1);
    c.launches++;
    return e;
  }
  if (var == 1) k_traverse<1><<<c.trav_grid, kThreads, 0, s>>>(t);
  else if (deep) k_traverse<kVarDeep><<<c.trav_grid, kThreads, 0, s>>>(t);
  else k_traverse<0><<<c.trav_grid, kThreads, 0, s>>>(t);
  e = cudaGetLastError();
  c.launches++;
  if (e) return e;
  k_order<false><<<c.num_sms * 4, kCostBuckets, 0, s>>>(c.d_counts, c.g_list, c.g_beg, nullptr, c.work_hist,
                                                        c.g_order);
  e = cudaGetLastError();
  c.launches++;
  if (e) return e;
  mark(0);
  if (var == 2) {
    if (mode == kOutSorted) k_eval_f64<kOutSorted><<<c.eval_grid, kThreads, 0, s>>>(a);
    else k_eval_f64<kOutCaller><<<c.eval_grid, kThreads, 0, s>>>(a);
    e = cudaGetLastError();
  } else
#define BH_EVAL_CASE(V, G, M) \
  if (var == V && guard == G && mode == M) e = launch_eval<V, G, M>(c, a, s); else
  BH_EVAL_CASE(0, false, kOutCaller)
  BH_EVAL_CASE(0, true, kOutCaller)
  BH_EVAL_CASE(0, false, kOutSorted)
  BH_EVAL_CASE(0, true, kOutSorted)
  BH_EVAL_CASE(1, false, kOutCaller)
  BH_EVAL_CASE(1, true, kOutCaller)
  BH_EVAL_CASE(1, false, kOutSorted)
  BH_EVAL_CASE(1, true, kOutSorted)
  BH_EVAL_CASE(kVarDeep, false, kOutCaller)
  BH_EVAL_CASE(kVarDeep, true, kOutCaller)
  BH_EVAL_CASE(kVarDeep, false, kOutSorted)
  BH_EVAL_CASE(kVarDeep, true, kOutSorted)
  e = cudaErrorInvalidValue;
#undef BH_EVAL_CASE
  mark(1);
  c.launches++;
  return e;
}

}  // namespace bh
