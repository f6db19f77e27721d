// k_noalloc.cu -- an exclusive prefix sum for callers that cannot allocate
// device memory.
//
// Some callers are not allowed to allocate GPU memory at all: a component
// that is handed device buffers by a host application which owns every
// byte of GPU memory (and accounts for it), or code that runs under a fixed
// device-memory budget set by someone else.  Such a caller cannot create a
// context and bind a workspace.  This entry point needs neither: its only
// scratch (the per-block sums of the scan) is a fixed array compiled into
// the library.
//
// The array lives in every GPU that loads the library until the process
// exits (128 KiB + 8 bytes: 16,384 64-bit block sums and the total).  Host code cannot use the array's name as a
// device address -- in host code it names a host-side stand-in -- so the
// first call on each device asks the runtime for the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it.
#include <cuda_runtime.h>

#include <mutex>

#include "bh_internal.cuh"

namespace {

constexpr int64_t kMaxN = BH_NOALLOC_SCAN_MAX_N;
constexpr int kMaxDevices = 64;

// 64-bit block sums of the largest scan (4096 values a block), then the total
constexpr int64_t kMaxBlocks = (kMaxN + 4095) / 4096;
static __device__ __align__(256) uint64_t g_scan_scratch[kMaxBlocks + 1];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scan_scratch on the current device (looked up once).
int scratch_on_current_device(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BH_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return BH_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BH_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BH_OK;
}

}  // namespace

extern "C" int bh_exclusive_scan_noalloc(const uint32_t *in_dev, uint32_t *out_dev, int64_t n, uint64_t *total_dev,
                                         void *stream) {
  if (n < 0) return BH_ERR_INVALID_ARG;
  if (n > kMaxN) return BH_ERR_CAPACITY;
  if (n > 0 && (!in_dev || !out_dev)) return BH_ERR_INVALID_ARG;
  if (bh::scan_blocks_for(n) > kMaxBlocks) return BH_ERR_CAPACITY;
  void *scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  uint64_t *blocks = static_cast<uint64_t *>(scratch);
  // the total goes to the caller's buffer, else to the array's last element
  uint64_t *total = total_dev ? total_dev : blocks + kMaxBlocks;
  cudaError_t e = bh::launch_scan_u32_raw(in_dev, out_dev, n, blocks, total, (cudaStream_t)stream);
  return e == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}
