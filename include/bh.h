/*
 * bh.h -- C ABI of the GB300 (sm_103a) sparse-octree gravitational tree-code.
 *
 * The library computes, on one GPU, the per-step force evaluation of the
 * Barnes-Hut tree-code of Bedorf, Gaburov & Portegies Zwart (arXiv:1106.1900):
 * Morton keys, radix sort, level-by-level sparse octree, monopole +
 * quadrupole moments, and the breadth-first group walk with the opening test
 * d > l/theta + delta (Eq. 1), followed by an FP64 leapfrog step (§3.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Units: G = 1 (N-body units).
 * - Layout: positions and velocities are [n][3] FP64, row-major; masses [n]
 *   FP64; accelerations [n][3] FP32; potentials [n] FP32.  Outputs are in the
 *   caller's input order.  n < 2^31.
 * - Memory: pointers named *_dev are CUDA device pointers, *_host are host
 *   pointers.  The caller owns every input and output buffer and the
 *   workspace.  After bh_bind_workspace the library never allocates device
 *   memory and never frees caller memory.
 * - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *   Calls are stream-ordered and asynchronous unless stated otherwise;
 *   input buffers must stay valid until the stream reaches the call.
 * - Errors: every call returns a bh_status_t code.  Nothing throws across the ABI.
 *   Errors detected on the device (non-finite input, a full walk stack, a
 *   bounded wait that gave up) are latched in a device status word that
 *   bh_status() returns after synchronising the stream.
 * - Threads: one context must not be used by two host threads at once.
 */
#ifndef BH_H
#define BH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bh_status_code {
    BH_OK = 0,
    BH_ERR_INVALID_ARG = 1, /* bad pointer, size, parameter or offsets */
    BH_ERR_CAPACITY = 2,    /* n or n_sys above the context's maxima, or a walk
                               stack, a group's list (split walk) or the list
                               pool overflowed (raise stack_capacity,
                               list_capacity, pool_per_body) */
    BH_ERR_NONFINITE = 3,   /* a position or mass is NaN or infinite */
    BH_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    BH_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    BH_ERR_STATE = 6,       /* call order violated (e.g. forces before build) */
    BH_ERR_NO_WORKSPACE = 7 /* no (or too small a) workspace is bound */
} bh_status_t;

/* Tunables (§2.1, §2.2).  Fill with bh_default_params, then override. */
typedef struct bh_params {
    int32_t n_leaf;         /* N_leaf: a cell with <= n_leaf bodies is a leaf (§2.1).
                               1..64, default 16. */
    int32_t n_crit;         /* N_crit: a group holds <= n_crit bodies (§2.2).
                               n_leaf..256, default 64 (groups of more than
                               64 bodies are evaluated in several passes). */
    int32_t stack_capacity; /* entries per breadth-first level stack of one walking
                               warp (§2.2 current/next-level stacks), default 16384 */
    int32_t walk_variant;   /* 0: FP32 in group-relative coordinates with compensated
                               accumulation across list tiles (default);
                               1: naive FP32 (absolute coordinates, plain sums);
                               2: FP64 evaluation (a slow precision reference) */
    int32_t walk_warps;     /* warps per walk block: 4 (the walk kernels are compiled for it) */
    int32_t walk_blocks_per_sm; /* persistent grids = SMs x this; 0 = occupancy */
    int32_t list_capacity;  /* split walk: longest cell list and longest particle
                               list of one group (§2.2 interaction lists),
                               default 16384 */
    int32_t pool_per_body;  /* interaction-list pool entries per body (the lists of
                               all groups of one walk, split walk only), default 768;
                               a pool above 2^34 entries (pool_per_body x n_max)
                               is refused with BH_ERR_CAPACITY at bh_create and
                               bh_workspace_bytes */
    int32_t walk_split;     /* 0: one fused kernel walks each group and evaluates its
                               lists from the walking warp's scratch (default);
                               1: a walk kernel writes every group's lists to the pool,
                               an evaluation kernel reads them (most expensive group
                               first).  Variant 2 always uses the split form.  Both
                               give bit-identical results. */
    int32_t mac;            /* opening criterion: 0: Eq. 1, d > l/theta + delta with d
                               from the cell's centre of mass to the group's box
                               (default); 1: the minimal-distance criterion (§2.3),
                               d > l/theta with d between the cell's cube and the
                               group's box (more interactions, smaller errors) */
    int32_t key_levels;     /* key depth D in levels, 20..30 (App. B).  20 (default):
                               the paper's 60-bit keys, trees at most 20 levels deep;
                               a level-20 cell holding more than n_leaf bodies stays
                               one leaf.  21..30: 3D-bit keys (a 60-bit word for
                               levels 1..20 and a second word for 21..D), bodies
                               quantised to 2^D cells per axis; the sort takes
                               ceil(3(D-20)/8) more digit passes and the workspace
                               24 B more per body.  Cells are identical to the 20-level
                               tree wherever no level-20 cell exceeds n_leaf. */
    int32_t list_buffer;    /* fused walk: entries of each of a walking warp's two
                               list buffers (cells, bodies), a multiple of 64 in
                               128..2^20, default 4096.  A buffer is evaluated
                               whenever it fills (§2.2, Fig. 3), so no list
                               length is limited. */
} bh_params;

typedef struct bh_ctx bh_ctx; /* opaque, library-owned host object */

/* Number of per-phase timers reported by bh_phase_times. */
#define BH_NPHASES 9
/* Phases: 0 frame+keys, 1 sort, 2 move, 3 cells+link+groups, 4 moments,
 *         5 walk (opening radii + traversal + evaluation), 6 leapfrog
 *         (predict+correct), 7 whole call, 8 the evaluation kernel alone
 *         (part of 5). */

/* Writes the defaults into *p.  Returns BH_OK or BH_ERR_INVALID_ARG (p NULL). */
int bh_default_params(bh_params *p);

/* Device workspace a context created with (p, n_max, n_sys_max) needs, in
 * bytes, written to *bytes.  The size grows linearly with n_max (cell table
 * bound D*floor(n/(n_leaf+1)) + n + n_sys, D = key_levels) plus the walk stacks
 * (SMs x resident warps x 2 x stack_capacity x 4 B) on `device`. */
int bh_workspace_bytes(const bh_params *p, int64_t n_max, int32_t n_sys_max, int device, size_t *bytes);

/* Creates a context for up to n_max bodies in up to n_sys_max systems on
 * `device` (made current for the call).  The context holds host state and
 * CUDA events only; device memory comes from bh_bind_workspace. */
int bh_create(bh_ctx **out, const bh_params *p, int64_t n_max, int32_t n_sys_max, int device);

/* Binds a caller-allocated device buffer of `bytes` >= bh_workspace_bytes(...)
 * (256-byte aligned).  The context keeps the pointer; the caller keeps
 * ownership and must keep it alive until bh_destroy. */
int bh_bind_workspace(bh_ctx *ctx, void *ws_dev, size_t bytes);

/* Destroys the context (host state, events and captured graphs). */
void bh_destroy(bh_ctx *ctx);

/* Builds the octree of one system (§2.1, App. B): frame and Morton keys,
 * stable radix sort, level-by-level cells, links, groups (§2.2) and the
 * monopole + quadrupole moments (§3.2).  pos_dev [n][3], mass_dev [n]. */
int bh_build(bh_ctx *ctx, const double *pos_dev, const double *mass_dev, int64_t n, void *stream);

/* The same for a forest of independent systems: system s owns bodies
 * sys_offsets_host[s] .. sys_offsets_host[s+1]-1 (ascending, [0] = 0,
 * [n_sys] = n; empty systems allowed).  Each system gets its own frame;
 * cells and groups never span two systems. */
int bh_build_forest(bh_ctx *ctx, const double *pos_dev, const double *mass_dev, int64_t n,
                    const int64_t *sys_offsets_host, int32_t n_sys, void *stream);

/* Accelerations and potentials of every body of the last build (§2.2, §3.3):
 * groups walk the tree breadth-first, accept cells with d^2 > (l/theta + delta)^2,
 * and sum softened particle-cell (monopole + quadrupole) and particle-particle
 * interactions in FP32.  theta > 0 (theta = 0 opens every cell), eps >= 0.
 * acc_dev [n][3], pot_dev [n], caller order. */
int bh_compute_forces(bh_ctx *ctx, float theta, float eps, float *acc_dev, float *pot_dev, void *stream);

/* The same round trip from host memory: copies pos/mass in, builds, walks,
 * copies acc/pot out, and synchronises the stream.  Host buffers should be
 * pinned for speed. */
int bh_forces_host(bh_ctx *ctx, const double *pos_host, const double *mass_host, int64_t n,
                   float theta, float eps, float *acc_host, float *pot_host, void *stream);

/* Loads the integrator state (FP64): n bodies, optional forest offsets
 * (sys_offsets_host NULL or n_sys <= 1 means one system).  The first bh_step
 * afterwards first evaluates the accelerations at the loaded positions. */
int bh_set_state(bh_ctx *ctx, const double *pos_dev, const double *vel_dev, const double *mass_dev, int64_t n,
                 const int64_t *sys_offsets_host, int32_t n_sys, void *stream);

/* Copies the state out in the order it was loaded; any pointer may be NULL.
 * acc/pot are the last evaluated accelerations and potentials. */
int bh_get_state(bh_ctx *ctx, double *pos_dev, double *vel_dev, float *acc_dev, float *pot_dev, void *stream);

/* One leapfrog predictor-corrector step (§3.1): x += v dt + a dt^2/2,
 * v_p = v + a dt, rebuild the tree at x, evaluate a_new, v = v_p +
 * (a_new - a) dt/2.  FP64 state, FP32 forces.  No host synchronisation. */
int bh_step(bh_ctx *ctx, double dt, float theta, float eps, void *stream);

/* bh_step through a CUDA graph: the first call with a given (dt, theta, eps)
 * captures one step on a context-owned stream and instantiates it; every
 * call then launches the graph on `stream`. */
int bh_step_graph(bh_ctx *ctx, double dt, float theta, float eps, void *stream);

/* ---- Block time-steps (the paper's motivation for an all-GPU tree code:
 * §1, the "active" groups of §2.2, moment refresh and rebuild of §4).  No
 * scheme is printed; the one built here: body i steps with dt_max 2^-k_i,
 * k_i in 0..k_max, on integer ticks of dt_max 2^-k_max; the level wanted is
 * the smallest k with dt_max 2^-k <= eta sqrt(eps / |a_i|).  A block step
 * advances to the earliest time T a body is due, predicts every body to T
 * (the bh_step predictor), rebuilds the tree at the predicted positions or
 * refreshes its moments on the unchanged tree (a cell keeps its geometric
 * centre and grows to the smallest cube about it holding its bodies or
 * children), walks only the groups holding a due body, and corrects the due
 * bodies (the bh_step corrector); a due body then takes a deeper level at
 * once, or one level shallower when T is a multiple of the doubled step.
 * With k_max = 0 a block step is a bh_step with dt = dt_max, bit for bit. */

/* Starts block time-stepping on the loaded state (bh_set_state): forces of
 * every body at t = 0, first levels, every body at tick 0.  eps > 0,
 * 0 <= k_max <= 40, dt_max > 0, eta > 0.  The state is left in the tree's
 * body order; bh_get_state still returns the caller's order. */
int bh_block_start(bh_ctx *ctx, double dt_max, int32_t k_max, double eta, float theta, float eps, void *stream);

/* One block step.  rebuild != 0 builds the tree anew at the predicted
 * positions; 0 refreshes the moments on the last tree (the first step after
 * bh_block_start may refresh).  BH_ERR_STATE without bh_block_start; a
 * bh_step, bh_set_state or bh_build ends block time-stepping. */
int bh_block_step(bh_ctx *ctx, float theta, float eps, int32_t rebuild, void *stream);

/* out[0] block time of the last step (ticks), out[1] bodies due at it,
 * out[2] groups walked, out[3] deepest level held after it.  Synchronises. */
int bh_block_info(bh_ctx *ctx, int64_t out[4], void *stream);

/* Each body's level (int32 [n]) and the tick of its last update (int64 [n]),
 * device buffers in the caller's order; either may be NULL. */
int bh_block_levels(bh_ctx *ctx, int32_t *level_dev, int64_t *tick_dev, void *stream);

/* A leapfrog step in three parts, for a system whose groups are shared out
 * among several GPUs (the paper's §5 names splitting the work over GPUs as
 * the way to larger systems; here the tree is built on every GPU and the
 * groups are split): every rank holds the whole state, builds the same tree,
 * walks only its own contiguous range of groups, exchanges the accelerations
 * of its groups' bodies with the other ranks (the caller's collective, e.g.
 * an all-gather over NCCL), and then corrects every body, so that all ranks
 * hold the same state again.
 *
 * bh_step_begin: the predictor (skipped with init = 1: the initial force
 *   evaluation at the loaded state, which must come first, once) and the
 *   build at the predicted positions.  Stream-ordered.
 * bh_walk_groups: the walk (§2.2) of groups g_begin <= g < g_end of that
 *   build (group order: bh_get_tree's gbeg), writing the accelerations and
 *   potentials of their bodies (sorted body range gbeg[g_begin] ..
 *   gend[g_end - 1]) into the context's sorted force array; may be called
 *   for several ranges.  g_end past the last group is clamped.  The walked
 *   groups' list statistics (bh_get_group_stats) are this walk's; the other
 *   groups' are left from earlier walks.
 * bh_sorted_forces: the device address of that array, float4 [n]
 *   (a.x, a.y, a.z, phi) in sorted body order, inside the bound workspace;
 *   the caller fills in the other ranks' body ranges before bh_step_end.
 * bh_step_end: the corrector of every body with the sorted force array
 *   (init as in bh_step_begin).
 * Out of order calls return BH_ERR_STATE.  Walking every group once and
 * calling bh_step_end gives exactly bh_step's result. */
int bh_step_begin(bh_ctx *ctx, double dt, int32_t init, void *stream);
int bh_walk_groups(bh_ctx *ctx, float theta, float eps, int32_t g_begin, int32_t g_end, void *stream);
int bh_sorted_forces(bh_ctx *ctx, float **acc_dev);
int bh_step_end(bh_ctx *ctx, double dt, int32_t init, void *stream);

/* Energies and momentum of the current state (FP64, synchronises):
 * out[0] kinetic, out[1] potential = 1/2 sum m phi, out[2..4] momentum.
 * The potentials are those of the last force evaluation. */
int bh_diagnostics(bh_ctx *ctx, double out[5], void *stream);

/* Synchronises `stream` and returns (and clears) the device status word. */
int bh_status(bh_ctx *ctx, void *stream);

/* Sizes of the last build (synchronises): out[0] n, out[1] cells, out[2]
 * groups, out[3] systems, out[4] deepest level, out[5] walk launches since
 * reset, out[6] particle-particle and out[7] particle-cell interactions summed
 * over those launches (self pairs excluded), out[8] kernel launches issued
 * by the library since reset. */
int bh_get_counts(bh_ctx *ctx, int64_t out[9], void *stream);

/* Failure detection test hook: runs the sort's bounded look-back wait on a
 * tile table that nothing publishes, so it gives up after spin_limit polls
 * (>= 1, capped at the library's own limit of 2^22) and latches
 * BH_ERR_TIMEOUT in the status word, which bh_status then returns (and
 * clears); the context stays usable.  Overwrites the sort's scratch and drops
 * captured step graphs.  BH_ERR_INVALID_ARG for spin_limit < 1. */
int bh_wait_probe(bh_ctx *ctx, int32_t spin_limit, void *stream);

/* Clears the interaction and launch counters of bh_get_counts. */
int bh_reset_counters(bh_ctx *ctx, void *stream);

/* Exports the integer tree of the last build to host arrays (synchronises);
 * any pointer may be NULL.  Sorted order: skey[n] 60-bit Morton keys, the
 * levels 1..20 of each key (a forest orders by system, then key; deeper
 * keys continue in bh_get_keys_lo), perm[n] input index of each sorted
 * body.  Cells (count from bh_get_counts) in (level, system, key) order:
 * level, pbeg, pend (sorted body range), parent (-1 at a root), first_child
 * (-1 at a leaf), n_children (0 at a leaf), is_leaf.  Groups in body order:
 * gbeg, gend. */
int bh_get_tree(bh_ctx *ctx, uint64_t *skey, int32_t *perm, int32_t *level, int32_t *pbeg, int32_t *pend,
                int32_t *parent, int32_t *first_child, int32_t *n_children, int32_t *is_leaf, int32_t *gbeg,
                int32_t *gend, void *stream);

/* Exports the low key words of the last build in sorted order (synchronises):
 * skey_lo[n] holds levels 21..D of each body's key (bit b of the low D-20
 * bits of q_x, q_y, q_z at bits 3b, 3b+1, 3b+2), all zero for key_levels =
 * 20; the full key is (skey << 3(D-20)) | skey_lo.  BH_ERR_INVALID_ARG for
 * a NULL pointer, BH_ERR_STATE before a build. */
int bh_get_keys_lo(bh_ctx *ctx, uint64_t *skey_lo, void *stream);

/* Exports the moments of every cell (synchronises), any pointer may be NULL:
 * mass[C], com[C][3] (FP64, recombined from its two-float form), quad[C][6]
 * (xx, yy, zz, xy, xz, yz, about the centre of mass), delta[C] =
 * |com - geometric centre|, size[C] = l. */
int bh_get_moments(bh_ctx *ctx, float *mass, double *com, float *quad, float *delta, float *size, void *stream);

/* Per-group statistics of the last walk (synchronises): cell-list length,
 * particle-list length, and the sums of the listed cell and body indices. */
int bh_get_group_stats(bh_ctx *ctx, int32_t *n_pc, int32_t *n_pp, uint64_t *csum, uint64_t *psum, void *stream);

/* Per-phase device times in milliseconds of the last bh_build +
 * bh_compute_forces or bh_step (see BH_NPHASES), recorded with CUDA events
 * when profiling is on (synchronises). */
int bh_set_profiling(bh_ctx *ctx, int on);
int bh_phase_times(bh_ctx *ctx, float ms[BH_NPHASES]);

/* Device time in milliseconds of the last walk phase alone (the opening-radius
 * pass and the walk kernel, phase 5), synchronising on it.  Profiling must be
 * on. */
int bh_walk_time(bh_ctx *ctx, float *ms);

/* App. A scan primitive (device-wide exclusive prefix sum of uint32), exposed
 * for verification: out_dev[i] = in_dev[0] + ... + in_dev[i-1] modulo 2^32,
 * and *total_host = the exact sum of all n values (synchronises).  Needs a bound
 * workspace and n <= n_max. */
int bh_prim_exclusive_scan(bh_ctx *ctx, const uint32_t *in_dev, uint32_t *out_dev, int64_t n, uint64_t *total_host,
                           void *stream);

/* The precision split of §3.2's reading (FP64 state, FP32 arithmetic in
 * cell-relative coordinates), exposed for verification: for i < n,
 * hi_dev[i] = x_dev[i] rounded to the nearest float (ties to even),
 * lo_dev[i] = x_dev[i] - hi_dev[i] (exact in FP64) rounded the same way, and
 * wide_dev[i] = f_dev[i] converted exactly to FP64 -- the conversions every
 * step applies to each body, done on the integer units.  All pointers are
 * device buffers of n elements owned by the caller.  No context needed;
 * stream-ordered, asynchronous.  Returns BH_ERR_INVALID_ARG for n < 0,
 * n >= 2^31 or a null pointer with n > 0, BH_ERR_CUDA if the launch fails. */
int bh_prim_split2(const double *x_dev, const float *f_dev, int64_t n, float *hi_dev, float *lo_dev,
                   double *wide_dev, void *stream);

/* Direct summation (§4.2.1 measures the tree's error against it; §3.3: theta
 * -> 0 turns the tree-code into it): acceleration and potential on each listed
 * target from every other body, softened like the particle-particle term.
 * pos_dev [n][3] FP64, mass_dev [n] FP64, targets_dev [nt] int32 body
 * indices; acc_dev [nt][3], pot_dev [nt] FP32 (pair differences from
 * two-float positions, TwoSum-folded tile sums).  No context needed;
 * stream-ordered.  O(nt * n) work: for subsamples and small systems. */
int bh_direct_forces(const double *pos_dev, const double *mass_dev, int64_t n, const int32_t *targets_dev,
                     int64_t nt, float eps, float *acc_dev, float *pot_dev, void *stream);

/* Exclusive prefix sum (the same operation as bh_prim_exclusive_scan) for
 * callers that cannot allocate device memory.  The paper has no counterpart:
 * this entry point exists for callers that are handed device buffers by an
 * application which owns all GPU memory, or that run under a device-memory
 * budget set by someone else, and so can neither allocate nor bind a
 * workspace.  It needs no context.
 *
 * in_dev[n], out_dev[n] (uint32, device): out_dev[i] = in_dev[0] + ... +
 * in_dev[i-1] modulo 2^32.  total_dev (device, may be NULL): receives the
 * exact sum of all n values as uint64 (0 for n = 0).  Stream-ordered, no host
 * synchronisation.
 *
 * Its only scratch is a fixed array compiled into the library (128 KiB +
 * 8 bytes), held by every GPU that loads the library until the process
 * exits.  It allocates nothing, so n is limited to BH_NOALLOC_SCAN_MAX_N:
 * larger n returns BH_ERR_CAPACITY before anything is launched.  The first
 * call on each device looks up the array's device address with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point again on a
 * device after cudaDeviceReset of that device (the kept address is then
 * stale).  Every call shares the one array (no call relies on what an
 * earlier call left in it), so calls that overlap on the GPU -- on
 * different streams, or from different host threads -- race: serialise
 * them. */
#define BH_NOALLOC_SCAN_MAX_N (1ll << 26)
int bh_exclusive_scan_noalloc(const uint32_t *in_dev, uint32_t *out_dev, int64_t n, uint64_t *total_dev,
                              void *stream);

/* A FP32 fused-multiply-add throughput probe: runs `iters` dependent FMA
 * chains on every resident thread and returns the achieved FP32 FLOP/s
 * (2 per FMA) in *flops.  Used to state the walk's FP32 roofline. */
int bh_fp32_peak_probe(int device, int iters, double *flops, void *stream);

/* Human-readable name of a status code (static string). */
const char *bh_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* BH_H */
