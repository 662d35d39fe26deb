// spk_noalloc.cu -- allocation-free column-pointer scan.
//
// The library's normal entry points allocate their workspace (stream-ordered
// or through the caller's allocator).  This file offers one entry point that
// allocates nothing: the exclusive scan of per-column counts into int64
// column pointers, with its per-tile partial sums kept in a fixed-size array
// that lives in this file for the life of the process.
#include <mutex>

#include "spkadd.h"
#include "spk_launch.h"

namespace {

// Scratch for the scan's tile sums plus the grand total.  SCAN_TILE = 4096
// counts per tile, so SPKADD_SCAN_NOALLOC_MAX_N counts need this many tiles.
constexpr int kNoallocTiles = SPKADD_SCAN_NOALLOC_MAX_N / 4096;
static __device__ __align__(256) long long g_scan_scratch[kNoallocTiles + 1];

std::mutex g_mu;
long long* g_addr[64];
bool g_have[64];

// Device address of g_scan_scratch on the current device, looked up once per
// device.  In host code the name g_scan_scratch is only a host-side stand-in,
// so kernels must be given this address instead.  The same first call loads
// the scan kernels' code onto the device (CUDA loads modules lazily, and a
// load takes device memory), so later calls load nothing.
cudaError_t scratch_address(long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_have[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scan_scratch);
    if (e == cudaSuccess) e = spk::load_scan_kernels();
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<long long*>(p);
    g_have[dev] = true;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) spkadd_status spkadd_scan_counts_noalloc(const int32_t* counts,
                                                                                           int64_t n,
                                                                                           int64_t* col_ptr,
                                                                                           void* stream) {
  if (!col_ptr || n < 0 || (n > 0 && !counts)) return SPKADD_ERR_INVALID_ARG;
  if (n > SPKADD_SCAN_NOALLOC_MAX_N) return SPKADD_ERR_UNSUPPORTED;
  long long* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e == cudaSuccess) e = spk::launch_scan(counts, (int)n, scratch, col_ptr, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) return SPKADD_OK;
  return e == cudaErrorMemoryAllocation ? SPKADD_ERR_NOMEM : SPKADD_ERR_CUDA;
}
