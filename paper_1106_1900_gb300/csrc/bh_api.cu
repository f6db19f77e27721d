// bh_api.cu -- the C ABI declared in include/bh.h: context and workspace,
// the per-step launch sequence, CUDA-graph capture, exports for parity checks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "bh_internal.cuh"

namespace bh {
int sort_passes_for(int S, int D);
int64_t sort_tiles_for(int64_t n);
}  // namespace bh

using bh::Ctx;

struct bh_ctx {
  Ctx c;
};

namespace {

constexpr size_t kAlign = 256;

int cu(cudaError_t e) { return e == cudaSuccess ? BH_OK : BH_ERR_CUDA; }

int validate_params(const bh_params *p) {
  if (!p) return BH_ERR_INVALID_ARG;
  if (p->n_leaf < 1 || p->n_leaf > 64) return BH_ERR_INVALID_ARG;
  if (p->n_crit < p->n_leaf || p->n_crit > bh::kMaxCrit) return BH_ERR_INVALID_ARG;
  if (p->stack_capacity < 64) return BH_ERR_INVALID_ARG;
  if (p->walk_variant < 0 || p->walk_variant > 2) return BH_ERR_INVALID_ARG;
  if (p->walk_warps != 4) return BH_ERR_INVALID_ARG;  // the walk kernels are compiled for 4-warp blocks
  if (p->walk_blocks_per_sm < 0 || p->walk_blocks_per_sm > 64) return BH_ERR_INVALID_ARG;
  if (p->list_capacity < 64 || p->pool_per_body < 1) return BH_ERR_INVALID_ARG;
  if (p->list_buffer < 128 || p->list_buffer > (1 << 20) || p->list_buffer % 64) return BH_ERR_INVALID_ARG;
  if (p->walk_split != 0 && p->walk_split != 1) return BH_ERR_INVALID_ARG;
  if (p->mac != 0 && p->mac != 1) return BH_ERR_INVALID_ARG;
  if (p->key_levels < bh::kLevels || p->key_levels > bh::kLevelsMax) return BH_ERR_INVALID_ARG;
  return BH_OK;
}

struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T *p = reinterpret_cast<T *>(base + off);
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

// Sizes that depend only on (params, n_max, n_sys_max, device).
int plan(Ctx &c, const bh_params *p, int64_t n_max, int32_t s_max, int device) {
  int rc = validate_params(p);
  if (rc) return rc;
  if (n_max < 1 || n_max >= (1ll << 30) || s_max < 1 || s_max > n_max + 1) return BH_ERR_INVALID_ARG;
  c.p = *p;
  c.device = device;
  c.n_max = n_max;
  c.s_max = s_max;
  c.levels = p->key_levels;
  c.c_max = (int64_t)c.levels * (n_max / (p->n_leaf + 1)) + n_max + s_max + 1;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return BH_ERR_CUDA;
  c.num_sms = prop.multiProcessorCount;
  c.walk_smem = bh::walk_smem_bytes(bh::walk_block_warps());
  int tb = p->walk_blocks_per_sm, eb = p->walk_blocks_per_sm, fb = p->walk_blocks_per_sm;
  {
    int dev0 = 0, t_occ = 1, e_occ = 1, f_occ = 1;
    cudaGetDevice(&dev0);
    cudaSetDevice(device);
    bh::walk_grids(&t_occ, &e_occ, &f_occ);
    cudaSetDevice(dev0);
    if (tb == 0) tb = t_occ;
    if (eb == 0) eb = e_occ;
    if (fb == 0) fb = f_occ;
  }
  // a small system needs fewer walking warps (each owns stack and list scratch)
  const int64_t want = std::max<int64_t>(c.num_sms, (n_max + 63) / 64);
  c.trav_grid = (int)std::min<int64_t>((int64_t)c.num_sms * tb, want);
  c.eval_grid = (int)std::min<int64_t>((int64_t)c.num_sms * eb, want);
  c.walk_grid = (int)std::min<int64_t>((int64_t)c.num_sms * fb, want);
  const bool fused = bh::walk_is_fused(*p);
  // (a walk of the active groups of a block step is always fused, so the split
  // form sizes its stacks and lists for both grids)
  c.trav_warps_total = (fused ? c.walk_grid : std::max(c.trav_grid, c.walk_grid)) * bh::walk_block_warps();
  // the list pool serves the split walk only
  c.pool_cap = fused ? 32 : std::max<int64_t>((int64_t)p->pool_per_body * n_max, 1ll << 22);
  // group offsets into the pool are stored as 32-bit multiples of kPoolAlign
  if (c.pool_cap > ((int64_t)bh::kPoolAlign << 32)) return BH_ERR_CAPACITY;
  c.sort_max_passes = bh::sort_passes_for(s_max, c.levels);
  c.sort_tiles_max = bh::sort_tiles_for(n_max);
  return BH_OK;
}

void carve(Ctx &c, char *base, size_t *total) {
  Carver k{base};
  const size_t N = (size_t)c.n_max, S = (size_t)c.s_max, C = (size_t)c.c_max;
  const size_t W = (N + 31) / 32;
  const size_t R = (size_t)(c.levels + 2) * W;
  c.offs = k.take<int32_t>(S + 1);
  c.minmax = k.take<unsigned long long>(6 * S);
  c.frame = k.take<bh::Frame>(S);
  c.framef = k.take<bh::FrameF>(S);
  c.sys_root = k.take<int32_t>(S);
  c.frame_ticket = k.take<uint32_t>(1);
  for (int b = 0; b < 2; ++b) {
    c.key[b] = k.take<uint64_t>(N);
    c.idx[b] = k.take<uint32_t>(N);
  }
  const bool deep = c.levels > bh::kLevels;
  c.key_hi0 = deep ? k.take<uint64_t>(N) : nullptr;
  c.key_lo0 = deep ? k.take<uint64_t>(N) : nullptr;
  c.skey_lo = deep ? k.take<uint64_t>(N) : nullptr;
  c.part_hi = k.take<float4>(N);
  c.part_lo = k.take<float4>(N);
  c.lohi = k.take<uint8_t>(2 * N);
  c.gstart = k.take<uint8_t>(N);
  c.acc_sorted = k.take<float4>(N);
  for (int b = 0; b < 2; ++b) {
    c.st_x[b] = k.take<double>(3 * N);
    c.st_v[b] = k.take<double>(3 * N);
    c.st_m[b] = k.take<double>(N);
    c.st_a[b] = k.take<float4>(N);
    c.st_id[b] = k.take<int32_t>(N);
    c.st_t[b] = k.take<int64_t>(N);
    c.st_k[b] = k.take<int32_t>(N);
  }
  c.h_pos = k.take<double>(3 * N);
  c.h_mass = k.take<double>(N);
  c.h_acc = k.take<float>(3 * N);
  c.h_pot = k.take<float>(N);
  c.rowcnt = k.take<uint32_t>(R + 1);
  c.rowoff = k.take<uint32_t>(R + 1);
  c.c_level = k.take<int32_t>(C);
  c.c_pbeg = k.take<int32_t>(C);
  c.c_pend = k.take<int32_t>(C);
  c.c_parent = k.take<int32_t>(C);
  c.c_first = k.take<int32_t>(C);
  c.c_nch = k.take<int32_t>(C);
  c.c_link = k.take<int2>(C);
  c.c_mom = k.take<float4>(4 * C);
  c.c_mac = k.take<float4>(C);
  c.c_mac_lo = deep ? k.take<float4>(C) : nullptr;
  c.g_beg = k.take<int32_t>(N + 1);
  c.g_sys = k.take<int32_t>(N);
  c.g_npc = k.take<int32_t>(N);
  c.g_npp = k.take<int32_t>(N);
  c.g_csum = k.take<unsigned long long>(N);
  c.g_psum = k.take<unsigned long long>(N);
  c.sort_hist = k.take<uint32_t>((size_t)c.sort_max_passes * 256);
  c.sort_status = k.take<uint32_t>((size_t)c.sort_max_passes * c.sort_tiles_max * 256);
  c.sort_tile_ctr = k.take<uint32_t>((size_t)c.sort_max_passes);
  c.scan_blocks = k.take<uint64_t>(std::max(R, N) / 4096 + 2);
  c.scan_total = k.take<uint64_t>(1);
  c.walk_stack = k.take<int32_t>((size_t)c.trav_warps_total * 2 * (size_t)c.p.stack_capacity);
  // the fused walk's bounded buffers, or the split walk's whole lists
  c.list_scratch = k.take<int32_t>((size_t)c.trav_warps_total * (size_t)bh::walk_list_stride(c.p));
  c.acc_hold = k.take<float4>(2 * N);
  c.list_pool = k.take<uint32_t>((size_t)c.pool_cap);
  c.pool_ctr = k.take<unsigned long long>(1);
  c.g_list = k.take<int4>(N);
  c.work_hist = k.take<uint32_t>(2 * bh::kCostBuckets);
  c.g_order = k.take<int32_t>(N);
  c.walk_queue = k.take<uint32_t>(2);
  c.d_counts = k.take<int32_t>(4);
  c.pred_x = k.take<double>(3 * N);
  c.pred_s = k.take<double>(3 * N);
  c.g_active = k.take<uint8_t>(N);
  c.d_block = k.take<unsigned long long>(4);
  c.d_totals = k.take<unsigned long long>(4);
  c.d_status = k.take<int32_t>(1);
  c.d_diag = k.take<double>(5 + 256 * 5);
  *total = k.off + kAlign;
}

// Event pair around one phase.  Inside a stream capture the records become
// event-record nodes of the graph (external records), so a replayed graph
// times its phases too.
void record(Ctx &c, cudaEvent_t e, cudaStream_t s) {
  if (c.capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

// Event slot of the leapfrog's predict (drift) kernel; phase 6 reports it
// with the correct (kick) kernel.
constexpr int kPhasePredict = BH_NPHASES;

struct Phase {
  Ctx &c;
  cudaStream_t s;
  int id;
  Phase(Ctx &c_, cudaStream_t s_, int id_) : c(c_), s(s_), id(id_) {
    if (c.profiling) record(c, c.ev[id][0], s);
  }
  ~Phase() {
    if (c.profiling) {
      record(c, c.ev[id][1], s);
      c.phase_rec[id] = true;
    }
  }
};

int ready(bh_ctx *ctx) {
  if (!ctx) return BH_ERR_INVALID_ARG;
  if (!ctx->c.ws) return BH_ERR_NO_WORKSPACE;
  return BH_OK;
}

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int now = 0;
    cudaGetDevice(&now);
    if (now != prev) cudaSetDevice(prev);
  }
};

int upload_offsets(Ctx &c, int64_t n, const int64_t *offs, int32_t S, cudaStream_t s) {
  std::vector<int32_t> h((size_t)S + 1);
  if (S <= 1 || !offs) {
    h.assign(2, 0);
    h[1] = (int32_t)n;
    S = 1;
  } else {
    if (offs[0] != 0 || offs[S] != n) return BH_ERR_INVALID_ARG;
    for (int32_t i = 0; i < S; ++i)
      if (offs[i + 1] < offs[i]) return BH_ERR_INVALID_ARG;
    for (int32_t i = 0; i <= S; ++i) h[i] = (int32_t)offs[i];
  }
  if (S > c.s_max) return BH_ERR_CAPACITY;
  c.n_sys = S;
  // a synchronous copy: the host vector dies with this call
  int rc = cu(cudaMemcpyAsync(c.offs, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, s));
  if (rc) return rc;
  return cu(cudaStreamSynchronize(s));
}

// keys, sort, cells, moments from positions/masses in [n][3] / [n] layout;
// the move permutes nothing (a plain build), the state, or the state with its
// block time-step ticks and levels (the tree's bodies then from pos)
enum Move { kMovePlain = 0, kMoveState = 1, kMoveBlock = 2 };
int build_pipeline(Ctx &c, const double *pos, const double *mass, Move move, cudaStream_t s) {
  cudaError_t e;
  {
    Phase ph(c, s, 0);
    if ((e = bh::launch_reset(c, s))) return cu(e);
    if ((e = bh::launch_frame_keys(c, pos, mass, s))) return cu(e);
  }
  {
    Phase ph(c, s, 1);
    if ((e = bh::launch_sort(c, s))) return cu(e);
  }
  {
    Phase ph(c, s, 2);
    if (move == kMoveBlock) e = bh::launch_move_block(c, s);
    else if (move == kMoveState) e = bh::launch_move_state(c, s);
    else e = bh::launch_move(c, pos, mass, s);
    if (e) return cu(e);
  }
  {
    Phase ph(c, s, 3);
    if ((e = bh::launch_cells(c, s))) return cu(e);
  }
  {
    Phase ph(c, s, 4);
    if ((e = bh::launch_moments(c, s))) return cu(e);
  }
  return BH_OK;
}

int walk_phase(Ctx &c, float theta, float eps, bh::OutMode mode, float *acc, float *pot, cudaStream_t s,
               const uint8_t *g_active = nullptr) {
  Phase ph(c, s, 5);
  cudaError_t e;
  if ((e = bh::launch_mac(c, theta, s))) return cu(e);
  if ((e = bh::launch_walk(c, theta, eps, mode, acc, pot, s, g_active))) return cu(e);
  return BH_OK;
}

int check_theta_eps(float theta, float eps) {
  if (!(theta >= 0.f) || !(eps >= 0.f) || !std::isfinite(eps) || !std::isfinite(theta)) return BH_ERR_INVALID_ARG;
  return BH_OK;
}

// One leapfrog step (init: evaluate the accelerations at the loaded state only).
int step_impl(Ctx &c, double dt, float theta, float eps, bool init, cudaStream_t s) {
  cudaError_t e;
  c.split_open = false;  // a whole step ends any step in parts
  if (c.n == 0) return BH_OK;
  if (!init) {
    Phase ph(c, s, kPhasePredict);
    if ((e = bh::launch_predict(c, dt, s))) return cu(e);
  }
  const int a = c.state_cur;
  int rc = build_pipeline(c, c.st_x[a], c.st_m[a], kMoveState, s);
  if (rc) return rc;
  rc = walk_phase(c, theta, eps, bh::kOutSorted, nullptr, nullptr, s);
  if (rc) return rc;
  {
    Phase ph(c, s, 6);
    if ((e = bh::launch_correct(c, init ? 0.0 : dt, s))) return cu(e);
  }
  c.built = true;
  c.forces = true;
  return BH_OK;
}

void drop_graphs(Ctx &c) {
  for (int p = 0; p < 2; ++p) {
    if (c.graph_exec[p]) cudaGraphExecDestroy(c.graph_exec[p]);
    if (c.graph[p]) cudaGraphDestroy(c.graph[p]);
    c.graph_exec[p] = nullptr;
    c.graph[p] = nullptr;
    c.graph_launches[p] = 0;
  }
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int bh_default_params(bh_params *p) {
  if (!p) return BH_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->n_leaf = 16;
  p->n_crit = 64;
  p->stack_capacity = 16384;
  p->walk_variant = 0;
  p->walk_warps = 4;
  p->walk_blocks_per_sm = 0;
  p->list_capacity = 16384;
  p->list_buffer = 4096;
  p->pool_per_body = 768;
  p->walk_split = 0;
  p->mac = 0;
  p->key_levels = bh::kLevels;
  return BH_OK;
}

int bh_workspace_bytes(const bh_params *p, int64_t n_max, int32_t n_sys_max, int device, size_t *bytes) {
  if (!bytes) return BH_ERR_INVALID_ARG;
  Ctx c;
  int rc = plan(c, p, n_max, n_sys_max, device);
  if (rc) return rc;
  carve(c, nullptr, bytes);
  return BH_OK;
}

int bh_create(bh_ctx **out, const bh_params *p, int64_t n_max, int32_t n_sys_max, int device) {
  if (!out) return BH_ERR_INVALID_ARG;
  *out = nullptr;
  bh_ctx *ctx = new (std::nothrow) bh_ctx();
  if (!ctx) return BH_ERR_CUDA;
  Ctx &c = ctx->c;
  int rc = plan(c, p, n_max, n_sys_max, device);
  if (rc) {
    delete ctx;
    return rc;
  }
  DeviceGuard g(device);
  carve(c, nullptr, &c.ws_bytes);
  for (int i = 0; i <= BH_NPHASES; ++i)
    for (int j = 0; j < 2; ++j)
      if (cudaEventCreate(&c.ev[i][j]) != cudaSuccess) {
        bh_destroy(ctx);
        return BH_ERR_CUDA;
      }
  if (bh::walk_init_attrs(c.walk_smem) != cudaSuccess || bh::build_init_attrs() != cudaSuccess) {
    bh_destroy(ctx);
    return BH_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    bh_destroy(ctx);
    return BH_ERR_CUDA;
  }
  *out = ctx;
  return BH_OK;
}

int bh_bind_workspace(bh_ctx *ctx, void *ws, size_t bytes) {
  if (!ctx || !ws) return BH_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  if (bytes < c.ws_bytes) return BH_ERR_NO_WORKSPACE;
  char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(ws) + kAlign - 1) / kAlign * kAlign);
  size_t total = 0;
  carve(c, base, &total);
  c.ws = reinterpret_cast<char *>(ws);
  DeviceGuard g(c.device);
  int rc = cu(cudaMemset(c.d_status, 0, sizeof(int32_t)));
  if (rc) return rc;
  rc = cu(cudaMemset(c.d_totals, 0, 4 * sizeof(unsigned long long)));
  if (rc) return rc;
  rc = cu(cudaMemset(c.d_counts, 0, 4 * sizeof(int32_t)));
  if (rc) return rc;
  c.built = c.forces = c.have_state = c.have_acc = false;
  drop_graphs(c);
  return BH_OK;
}

void bh_destroy(bh_ctx *ctx) {
  if (!ctx) return;
  Ctx &c = ctx->c;
  DeviceGuard g(c.device);
  drop_graphs(c);
  for (int i = 0; i <= BH_NPHASES; ++i)
    for (int j = 0; j < 2; ++j)
      if (c.ev[i][j]) cudaEventDestroy(c.ev[i][j]);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  delete ctx;
}

static int build_common(bh_ctx *ctx, const double *pos, const double *mass, int64_t n, const int64_t *offs,
                        int32_t S, cudaStream_t s) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (n < 0 || (n > 0 && (!pos || !mass))) return BH_ERR_INVALID_ARG;
  if (n > c.n_max) return BH_ERR_CAPACITY;
  DeviceGuard g(c.device);
  rc = upload_offsets(c, n, offs, S, s);
  if (rc) return rc;
  c.n = n;
  c.built = c.forces = false;
  c.have_state = c.have_acc = false;
  c.block_on = c.block_tree = false;
  drop_graphs(c);
  for (int i = 0; i <= BH_NPHASES; ++i) c.phase_rec[i] = false;
  if (c.profiling) cudaEventRecord(c.ev[7][0], s);
  if (n == 0) {
    rc = cu(cudaMemsetAsync(c.d_counts, 0, 4 * sizeof(int32_t), s));
  } else {
    rc = build_pipeline(c, pos, mass, kMovePlain, s);
  }
  if (c.profiling) {
    cudaEventRecord(c.ev[7][1], s);
    c.phase_rec[7] = true;
  }
  if (rc) return rc;
  c.built = true;
  return BH_OK;
}

int bh_build(bh_ctx *ctx, const double *pos, const double *mass, int64_t n, void *stream) {
  return build_common(ctx, pos, mass, n, nullptr, 1, (cudaStream_t)stream);
}

int bh_build_forest(bh_ctx *ctx, const double *pos, const double *mass, int64_t n, const int64_t *offs,
                    int32_t n_sys, void *stream) {
  if (n_sys < 1 || !offs) return BH_ERR_INVALID_ARG;
  return build_common(ctx, pos, mass, n, offs, n_sys, (cudaStream_t)stream);
}

int bh_compute_forces(bh_ctx *ctx, float theta, float eps, float *acc, float *pot, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.built || c.have_state) return BH_ERR_STATE;
  rc = check_theta_eps(theta, eps);
  if (rc) return rc;
  if (c.n > 0 && (!acc || !pot)) return BH_ERR_INVALID_ARG;
  if (c.n == 0) return BH_OK;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  if (c.profiling) cudaEventRecord(c.ev[7][0], s);
  for (int i = 0; i <= BH_NPHASES; ++i) c.phase_rec[i] = false;
  rc = walk_phase(c, theta, eps, bh::kOutCaller, acc, pot, s);
  if (c.profiling) {
    cudaEventRecord(c.ev[7][1], s);
    c.phase_rec[7] = true;
  }
  if (rc) return rc;
  c.forces = true;
  return BH_OK;
}

int bh_forces_host(bh_ctx *ctx, const double *pos, const double *mass, int64_t n, float theta, float eps,
                   float *acc, float *pot, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (n < 0 || n > c.n_max) return n < 0 ? BH_ERR_INVALID_ARG : BH_ERR_CAPACITY;
  if (n > 0 && (!pos || !mass || !acc || !pot)) return BH_ERR_INVALID_ARG;
  rc = check_theta_eps(theta, eps);
  if (rc) return rc;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    if ((rc = cu(cudaMemcpyAsync(c.h_pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s)))) return rc;
    if ((rc = cu(cudaMemcpyAsync(c.h_mass, mass, sizeof(double) * n, cudaMemcpyHostToDevice, s)))) return rc;
  }
  rc = build_common(ctx, c.h_pos, c.h_mass, n, nullptr, 1, s);
  if (rc) return rc;
  if (n > 0) {
    rc = walk_phase(c, theta, eps, bh::kOutCaller, c.h_acc, c.h_pot, s);
    if (rc) return rc;
    if ((rc = cu(cudaMemcpyAsync(acc, c.h_acc, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s)))) return rc;
    if ((rc = cu(cudaMemcpyAsync(pot, c.h_pot, sizeof(float) * n, cudaMemcpyDeviceToHost, s)))) return rc;
  }
  c.forces = true;
  return cu(cudaStreamSynchronize(s));
}

int bh_set_state(bh_ctx *ctx, const double *pos, const double *vel, const double *mass, int64_t n,
                 const int64_t *offs, int32_t n_sys, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (n < 0 || (n > 0 && (!pos || !vel || !mass))) return BH_ERR_INVALID_ARG;
  if (n > c.n_max) return BH_ERR_CAPACITY;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  rc = upload_offsets(c, n, (n_sys > 1) ? offs : nullptr, (n_sys > 1) ? n_sys : 1, s);
  if (rc) return rc;
  c.n = n;
  c.state_cur = 0;
  drop_graphs(c);
  c.built = c.forces = false;
  c.block_on = c.block_tree = false;
  if (n > 0) {
    cudaError_t e = bh::launch_load_state(c, pos, vel, mass, s);
    if (e) return cu(e);
  }
  c.have_state = true;
  c.have_acc = false;
  return BH_OK;
}

int bh_get_state(bh_ctx *ctx, double *pos, double *vel, float *acc, float *pot, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.have_state) return BH_ERR_STATE;
  if (c.n == 0) return BH_OK;
  DeviceGuard g(c.device);
  return cu(bh::launch_get_state(c, pos, vel, acc, pot, (cudaStream_t)stream));
}

int bh_step(bh_ctx *ctx, double dt, float theta, float eps, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.have_state) return BH_ERR_STATE;
  rc = check_theta_eps(theta, eps);
  if (rc) return rc;
  if (!std::isfinite(dt)) return BH_ERR_INVALID_ARG;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  c.block_on = c.block_tree = false;  // a shared step moves every body by dt
  for (int i = 0; i <= BH_NPHASES; ++i) c.phase_rec[i] = false;
  if (c.profiling) cudaEventRecord(c.ev[7][0], s);
  if (!c.have_acc) {
    rc = step_impl(c, 0.0, theta, eps, true, s);
    if (rc) return rc;
    c.have_acc = true;
  }
  rc = step_impl(c, dt, theta, eps, false, s);
  if (c.profiling) {
    cudaEventRecord(c.ev[7][1], s);
    c.phase_rec[7] = true;
  }
  return rc;
}

int bh_step_graph(bh_ctx *ctx, double dt, float theta, float eps, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.have_state) return BH_ERR_STATE;
  rc = check_theta_eps(theta, eps);
  if (rc) return rc;
  if (!std::isfinite(dt)) return BH_ERR_INVALID_ARG;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  c.block_on = c.block_tree = false;  // a shared step moves every body by dt
  if (!c.have_acc) {
    rc = step_impl(c, 0.0, theta, eps, true, s);
    if (rc) return rc;
    c.have_acc = true;
  }
  if (c.n == 0) return BH_OK;
  if (c.g_dt != dt || c.g_theta != theta || c.g_eps != eps) {
    drop_graphs(c);
    c.g_dt = dt;
    c.g_theta = theta;
    c.g_eps = eps;
  }
  const int par = c.state_cur;
  if (!c.graph_exec[par]) {
    // capture one step from this buffer parity on the context's own stream;
    // the host bookkeeping (state_cur) advances during the capture
    const long long before = c.launches;
    if ((rc = cu(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal)))) return rc;
    c.capturing = true;
    int rs = step_impl(c, dt, theta, eps, false, c.cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c.cap_stream, &graph);
    c.capturing = false;
    if (rs || ee) {
      if (graph) cudaGraphDestroy(graph);
      c.state_cur = par;
      return rs ? rs : cu(ee);
    }
    c.graph[par] = graph;
    c.graph_launches[par] = c.launches - before;
    c.launches = before;
    if ((rc = cu(cudaGraphInstantiate(&c.graph_exec[par], graph, 0)))) {
      c.state_cur = par;
      return rc;
    }
  } else {
    c.state_cur = par ^ 1;
  }
  c.launches += c.graph_launches[par];
  return cu(cudaGraphLaunch(c.graph_exec[par], s));
}

int bh_step_begin(bh_ctx *ctx, double dt, int32_t init, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.have_state) return BH_ERR_STATE;
  if (!std::isfinite(dt) || (init != 0 && init != 1)) return BH_ERR_INVALID_ARG;
  if (!init && !c.have_acc) return BH_ERR_STATE;  // the accelerations at the loaded state come first
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  c.block_on = c.block_tree = false;
  c.split_open = false;
  if (c.n == 0) {
    c.split_open = true;
    c.split_init = init;
    return BH_OK;
  }
  cudaError_t e;
  if (!init) {
    Phase ph(c, s, kPhasePredict);
    if ((e = bh::launch_predict(c, dt, s))) return cu(e);
  }
  const int a = c.state_cur;
  if ((rc = build_pipeline(c, c.st_x[a], c.st_m[a], kMoveState, s))) return rc;
  c.built = true;
  c.split_open = true;
  c.split_init = init;
  return BH_OK;
}

int bh_walk_groups(bh_ctx *ctx, float theta, float eps, int32_t g_begin, int32_t g_end, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.split_open) return BH_ERR_STATE;
  if ((rc = check_theta_eps(theta, eps))) return rc;
  if (g_begin < 0 || g_end < g_begin) return BH_ERR_INVALID_ARG;
  if (c.n == 0 || g_end == g_begin) return BH_OK;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = bh::launch_mark_groups(c, g_begin, g_end, s))) return cu(e);
  if ((rc = walk_phase(c, theta, eps, bh::kOutSorted, nullptr, nullptr, s, c.g_active))) return rc;
  c.forces = true;  // (the walked groups' statistics are exported by bh_get_group_stats)
  return BH_OK;
}

int bh_sorted_forces(bh_ctx *ctx, float **acc_dev) {
  int rc = ready(ctx);
  if (rc) return rc;
  if (!acc_dev) return BH_ERR_INVALID_ARG;
  *acc_dev = reinterpret_cast<float *>(ctx->c.acc_sorted);
  return BH_OK;
}

int bh_step_end(bh_ctx *ctx, double dt, int32_t init, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.split_open) return BH_ERR_STATE;
  if (init != c.split_init || !std::isfinite(dt)) return BH_ERR_INVALID_ARG;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  c.split_open = false;
  if (init) c.have_acc = true;
  if (c.n == 0) return BH_OK;
  {
    Phase ph(c, s, 6);
    cudaError_t e = bh::launch_correct(c, init ? 0.0 : dt, s);
    if (e) return cu(e);
  }
  c.forces = true;
  return BH_OK;
}

int bh_block_start(bh_ctx *ctx, double dt_max, int32_t k_max, double eta, float theta, float eps, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.have_state) return BH_ERR_STATE;
  rc = check_theta_eps(theta, eps);
  if (rc) return rc;
  if (!(eps > 0.f) || !(dt_max > 0.0) || !std::isfinite(dt_max) || !(eta > 0.0) || !std::isfinite(eta) ||
      k_max < 0 || k_max > 40)
    return BH_ERR_INVALID_ARG;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  c.block_on = c.block_tree = false;
  c.blk_dt_max = dt_max;
  c.blk_kmax = k_max;
  c.blk_eta = eta;
  c.blk_tick = std::ldexp(dt_max, -k_max);
  if (c.n == 0) {
    c.block_on = true;
    return BH_OK;
  }
  // forces at t = 0 for every body (the state is left in the tree's body order)
  rc = step_impl(c, 0.0, theta, eps, true, s);
  if (rc) return rc;
  c.have_acc = true;
  if ((rc = cu(bh::launch_block_levels(c, (double)eps, s)))) return rc;
  c.block_on = c.block_tree = true;
  return BH_OK;
}

int bh_block_step(bh_ctx *ctx, float theta, float eps, int32_t rebuild, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.block_on) return BH_ERR_STATE;
  rc = check_theta_eps(theta, eps);
  if (rc) return rc;
  if (!(eps > 0.f)) return BH_ERR_INVALID_ARG;
  if (c.n == 0) return BH_OK;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  drop_graphs(c);
  for (int i = 0; i <= BH_NPHASES; ++i) c.phase_rec[i] = false;
  if (c.profiling) cudaEventRecord(c.ev[7][0], s);
  const bool full = rebuild || !c.block_tree;
  cudaError_t e;
  {
    Phase ph(c, s, kPhasePredict);
    if ((e = bh::launch_block_predict(c, s))) return cu(e);
  }
  if (full) {
    rc = build_pipeline(c, c.pred_x, c.st_m[c.state_cur], kMoveBlock, s);
    if (rc) return rc;
  } else {
    {
      Phase ph(c, s, 2);
      if ((e = bh::launch_block_parts(c, s))) return cu(e);
    }
    Phase ph(c, s, 4);
    if ((e = bh::launch_moments_refresh(c, s))) return cu(e);
  }
  if ((e = bh::launch_group_active(c, s))) return cu(e);
  rc = walk_phase(c, theta, eps, bh::kOutSorted, nullptr, nullptr, s, c.g_active);
  if (rc) return rc;
  {
    Phase ph(c, s, 6);
    if ((e = bh::launch_block_correct(c, (double)eps, full, s))) return cu(e);
  }
  if (c.profiling) {
    cudaEventRecord(c.ev[7][1], s);
    c.phase_rec[7] = true;
  }
  c.built = c.forces = c.block_tree = true;
  return BH_OK;
}

int bh_block_info(bh_ctx *ctx, int64_t out[4], void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!out) return BH_ERR_INVALID_ARG;
  if (!c.block_on) return BH_ERR_STATE;
  for (int q = 0; q < 4; ++q) out[q] = 0;
  if (c.n == 0) return BH_OK;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long b[4];
  int32_t cnt[4];
  if ((rc = cu(cudaMemcpyAsync(b, c.d_block, sizeof(b), cudaMemcpyDeviceToHost, s)))) return rc;
  if ((rc = cu(cudaMemcpyAsync(cnt, c.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost, s)))) return rc;
  if ((rc = cu(cudaStreamSynchronize(s)))) return rc;
  out[0] = (int64_t)b[0];
  out[1] = (int64_t)b[1];
  out[2] = (int64_t)cnt[3];
  out[3] = (int64_t)b[2];
  return BH_OK;
}

int bh_block_levels(bh_ctx *ctx, int32_t *level, int64_t *tick, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.block_on) return BH_ERR_STATE;
  if (c.n == 0) return BH_OK;
  DeviceGuard g(c.device);
  return cu(bh::launch_block_get(c, level, tick, (cudaStream_t)stream));
}

int bh_diagnostics(bh_ctx *ctx, double out[5], void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!out) return BH_ERR_INVALID_ARG;
  if (!c.have_state) return BH_ERR_STATE;
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  if (c.n == 0) return BH_OK;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = bh::launch_diag(c, s);
  if (e) return cu(e);
  if ((rc = cu(cudaMemcpyAsync(out, c.d_diag, 5 * sizeof(double), cudaMemcpyDeviceToHost, s)))) return rc;
  return cu(cudaStreamSynchronize(s));
}

int bh_status(bh_ctx *ctx, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = cu(cudaStreamSynchronize(s)))) return rc;
  int32_t st = 0;
  if ((rc = cu(cudaMemcpy(&st, c.d_status, sizeof(st), cudaMemcpyDeviceToHost)))) return rc;
  if (st) {
    if ((rc = cu(cudaMemset(c.d_status, 0, sizeof(int32_t))))) return rc;
  }
  return st;
}

int bh_wait_probe(bh_ctx *ctx, int32_t spin_limit, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  if (spin_limit < 1) return BH_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  DeviceGuard g(c.device);
  drop_graphs(c);  // the probe reuses the sort's tile table
  return cu(bh::launch_wait_probe(c, spin_limit, (cudaStream_t)stream));
}

int bh_get_counts(bh_ctx *ctx, int64_t out[9], void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  if (!out) return BH_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  DeviceGuard g(c.device);
  if ((rc = cu(cudaStreamSynchronize((cudaStream_t)stream)))) return rc;
  int32_t cnt[4] = {0, 0, 0, 0};
  unsigned long long tot[4] = {0, 0, 0, 0};
  if ((rc = cu(cudaMemcpy(cnt, c.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost)))) return rc;
  if ((rc = cu(cudaMemcpy(tot, c.d_totals, sizeof(tot), cudaMemcpyDeviceToHost)))) return rc;
  int deepest = -1;
  if (c.n > 0 && c.built) {
    const size_t W = (size_t)(c.n + 31) / 32;
    uint32_t starts[bh::kRowsMax];
    if ((rc = cu(cudaMemcpy2D(starts, sizeof(uint32_t), c.rowoff, W * sizeof(uint32_t), sizeof(uint32_t),
                              c.levels + 2, cudaMemcpyDeviceToHost))))
      return rc;
    for (int k = 0; k <= c.levels; ++k) {
      uint32_t next = starts[k + 1];
      if (next > starts[k]) deepest = k;
    }
  }
  out[0] = c.n;
  out[1] = c.built ? cnt[0] : 0;
  out[2] = c.built ? cnt[1] : 0;
  out[3] = c.n_sys;
  out[4] = deepest;
  out[5] = (int64_t)tot[2];
  out[6] = (int64_t)tot[0];
  out[7] = (int64_t)tot[1];
  out[8] = c.launches;
  return BH_OK;
}

int bh_reset_counters(bh_ctx *ctx, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  DeviceGuard g(c.device);
  c.launches = 0;
  return cu(cudaMemsetAsync(c.d_totals, 0, 4 * sizeof(unsigned long long), (cudaStream_t)stream));
}

int bh_get_tree(bh_ctx *ctx, uint64_t *skey, int32_t *perm, int32_t *level, int32_t *pbeg, int32_t *pend,
                int32_t *parent, int32_t *first_child, int32_t *n_children, int32_t *is_leaf, int32_t *gbeg,
                int32_t *gend, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.built) return BH_ERR_STATE;
  DeviceGuard g(c.device);
  if ((rc = cu(cudaStreamSynchronize((cudaStream_t)stream)))) return rc;
  int32_t cnt[4];
  if ((rc = cu(cudaMemcpy(cnt, c.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost)))) return rc;
  const size_t n = (size_t)c.n, C = (size_t)cnt[0], G = (size_t)cnt[1];
  auto get = [&](void *dst, const void *src, size_t bytes) -> int {
    if (!dst || bytes == 0) return BH_OK;
    return cu(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  };
  if ((rc = get(skey, c.key[0], n * 8))) return rc;
  if ((rc = get(perm, c.idx[0], n * 4))) return rc;
  if (level || is_leaf) {
    std::vector<int32_t> lv(C);
    if ((rc = get(lv.data(), c.c_level, C * 4))) return rc;
    for (size_t i = 0; i < C; ++i) {
      if (level) level[i] = lv[i] & 31;
      if (is_leaf) is_leaf[i] = (lv[i] >> 5) & 1;
    }
  }
  if ((rc = get(pbeg, c.c_pbeg, C * 4))) return rc;
  if ((rc = get(pend, c.c_pend, C * 4))) return rc;
  if ((rc = get(parent, c.c_parent, C * 4))) return rc;
  if ((rc = get(first_child, c.c_first, C * 4))) return rc;
  if ((rc = get(n_children, c.c_nch, C * 4))) return rc;
  if ((rc = get(gbeg, c.g_beg, G * 4))) return rc;
  if ((rc = get(gend, c.g_beg + 1, G * 4))) return rc;
  return BH_OK;
}

int bh_get_keys_lo(bh_ctx *ctx, uint64_t *skey_lo, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.built) return BH_ERR_STATE;
  if (!skey_lo) return BH_ERR_INVALID_ARG;
  DeviceGuard g(c.device);
  if ((rc = cu(cudaStreamSynchronize((cudaStream_t)stream)))) return rc;
  const size_t n = (size_t)c.n;
  if (!c.skey_lo) {
    std::memset(skey_lo, 0, n * sizeof(uint64_t));
    return BH_OK;
  }
  return n ? cu(cudaMemcpy(skey_lo, c.skey_lo, n * sizeof(uint64_t), cudaMemcpyDeviceToHost)) : BH_OK;
}

int bh_get_moments(bh_ctx *ctx, float *mass, double *com, float *quad, float *delta, float *size, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.built) return BH_ERR_STATE;
  DeviceGuard g(c.device);
  if ((rc = cu(cudaStreamSynchronize((cudaStream_t)stream)))) return rc;
  int32_t cnt[4];
  if ((rc = cu(cudaMemcpy(cnt, c.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost)))) return rc;
  const size_t C = (size_t)cnt[0];
  std::vector<float4> m(4 * C);
  if (C && (rc = cu(cudaMemcpy(m.data(), c.c_mom, sizeof(float4) * 4 * C, cudaMemcpyDeviceToHost)))) return rc;
  for (size_t i = 0; i < C; ++i) {
    const float4 a = m[4 * i], b = m[4 * i + 1], q0 = m[4 * i + 2], q1 = m[4 * i + 3];
    if (mass) mass[i] = a.w;
    if (com) {
      com[3 * i] = (double)a.x + (double)b.x;
      com[3 * i + 1] = (double)a.y + (double)b.y;
      com[3 * i + 2] = (double)a.z + (double)b.z;
    }
    if (quad) {
      quad[6 * i] = q0.x;
      quad[6 * i + 1] = q0.y;
      quad[6 * i + 2] = q0.z;
      quad[6 * i + 3] = q0.w;
      quad[6 * i + 4] = q1.x;
      quad[6 * i + 5] = q1.y;
    }
    if (delta) delta[i] = b.w;
    if (size) size[i] = q1.z;
  }
  return BH_OK;
}

int bh_get_group_stats(bh_ctx *ctx, int32_t *n_pc, int32_t *n_pp, uint64_t *csum, uint64_t *psum, void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (!c.forces) return BH_ERR_STATE;
  DeviceGuard g(c.device);
  if ((rc = cu(cudaStreamSynchronize((cudaStream_t)stream)))) return rc;
  int32_t cnt[4];
  if ((rc = cu(cudaMemcpy(cnt, c.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost)))) return rc;
  const size_t G = (size_t)cnt[1];
  if (G == 0) return BH_OK;
  if (n_pc && (rc = cu(cudaMemcpy(n_pc, c.g_npc, G * 4, cudaMemcpyDeviceToHost)))) return rc;
  if (n_pp && (rc = cu(cudaMemcpy(n_pp, c.g_npp, G * 4, cudaMemcpyDeviceToHost)))) return rc;
  if (csum && (rc = cu(cudaMemcpy(csum, c.g_csum, G * 8, cudaMemcpyDeviceToHost)))) return rc;
  if (psum && (rc = cu(cudaMemcpy(psum, c.g_psum, G * 8, cudaMemcpyDeviceToHost)))) return rc;
  return BH_OK;
}

int bh_set_profiling(bh_ctx *ctx, int on) {
  if (!ctx) return BH_ERR_INVALID_ARG;
  ctx->c.profiling = on != 0;
  return BH_OK;
}

int bh_phase_times(bh_ctx *ctx, float ms[BH_NPHASES]) {
  if (!ctx || !ms) return BH_ERR_INVALID_ARG;
  Ctx &c = ctx->c;
  DeviceGuard g(c.device);
  // slot BH_NPHASES holds the predict half of the leapfrog, reported in phase 6
  float t[BH_NPHASES + 1];
  for (int i = 0; i <= BH_NPHASES; ++i) {
    t[i] = 0.f;
    if (!c.phase_rec[i]) continue;
    if (cudaEventSynchronize(c.ev[i][1]) != cudaSuccess) return BH_ERR_CUDA;
    if (cudaEventElapsedTime(&t[i], c.ev[i][0], c.ev[i][1]) != cudaSuccess) {
      t[i] = 0.f;
      cudaGetLastError();  // do not leave the failed query for the next launch check
    }
  }
  for (int i = 0; i < BH_NPHASES; ++i) ms[i] = t[i];
  ms[6] += t[kPhasePredict];
  return BH_OK;
}

int bh_walk_time(bh_ctx *ctx, float *ms) {
  if (!ctx || !ms) return BH_ERR_INVALID_ARG;
  float all[BH_NPHASES];
  int rc = bh_phase_times(ctx, all);
  *ms = all[5];
  return rc;
}

int bh_prim_exclusive_scan(bh_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n, uint64_t *total,
                           void *stream) {
  int rc = ready(ctx);
  if (rc) return rc;
  Ctx &c = ctx->c;
  if (n < 0 || (n > 0 && (!in || !out)) || !total) return BH_ERR_INVALID_ARG;
  if (n > c.n_max) return BH_ERR_CAPACITY;
  DeviceGuard g(c.device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = bh::launch_scan_u32(c, in, out, n, s);
  if (e) return cu(e);
  if ((rc = cu(cudaMemcpyAsync(total, c.scan_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s)))) return rc;
  return cu(cudaStreamSynchronize(s));
}

int bh_fp32_peak_probe(int device, int iters, double *flops, void *stream) {
  if (!flops || iters < 1) return BH_ERR_INVALID_ARG;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return BH_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 256;
  const int blocks = prop.multiProcessorCount * (prop.maxThreadsPerMultiProcessor / threads);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) || cudaEventCreate(&b)) return BH_ERR_CUDA;
  bh::launch_fma_probe(blocks, threads, iters, nullptr, s);  // warm-up
  cudaEventRecord(a, s);
  bh::launch_fma_probe(blocks, threads, iters, nullptr, s);
  cudaEventRecord(b, s);
  int rc = cu(cudaEventSynchronize(b));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  *flops = (double)blocks * threads * (double)iters * 16.0 * 8.0 * 2.0 / (ms * 1e-3);
  return BH_OK;
}

const char *bh_status_string(int st) {
  switch (st) {
    case BH_OK: return "ok";
    case BH_ERR_INVALID_ARG: return "invalid argument";
    case BH_ERR_CAPACITY: return "capacity exceeded";
    case BH_ERR_NONFINITE: return "non-finite input";
    case BH_ERR_TIMEOUT: return "bounded device wait gave up";
    case BH_ERR_CUDA: return "CUDA runtime error";
    case BH_ERR_STATE: return "call order violated";
    case BH_ERR_NO_WORKSPACE: return "no or too small workspace bound";
    default: return "unknown status";
  }
}

}  // extern "C"
