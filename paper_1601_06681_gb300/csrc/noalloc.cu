// Allocation-free variant of the FP64 trace residual (ehdg_trace_residual).
//
// Some callers cannot allocate device memory: code that runs under a host
// application's memory manager, which owns every device allocation and its
// budget, and code in latency-critical loops where cudaMalloc/cudaFree would
// synchronise the device. For them the block partial sums live in this
// file-scope device array instead of in memory allocated per call. Every GPU
// that loads the library holds the array until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ehdg_internal.h"

namespace {

constexpr int kNoAllocMaxBlocks = 1024;         // block partial sums held by the array
static_assert(kNoAllocMaxBlocks >= ehdg::kResidMaxBlocks,
              "the array must hold a partial sum for every block the residual kernel launches");
constexpr int kNoAllocMaxDevices = 64;
// one partial per block plus the last-block ticket
constexpr size_t kNoAllocScratchBytes = sizeof(double) * kNoAllocMaxBlocks + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the array on the current device. In host code the
// array's name is only a host-side stand-in, so its device address is looked
// up once per device, with that device current, and kept for the life of the
// process (a cudaDeviceReset between calls would leave it stale, and is not
// supported).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ehdg_status ehdg_trace_residual_noalloc(const double* a, const double* b,
                                                   const double* w, int64_t n, double* out,
                                                   void* stream) {
  using namespace ehdg;
  if (!out || n < 0 || (n > 0 && (!a || !b || !w))) {
    set_last_error("ehdg_trace_residual_noalloc: NULL pointer or negative size");
    return EHDG_ERR_INVALID;
  }
  if (n > EHDG_NOALLOC_MAX_N) {
    set_last_error("ehdg_trace_residual_noalloc: n = " + std::to_string(n) +
                   " exceeds the maximum of " + std::to_string((long long)EHDG_NOALLOC_MAX_N) +
                   " entries this allocation-free entry point accepts");
    return EHDG_ERR_UNSUPPORTED;
  }
  if (wdiff_norm_blocks(n) > kNoAllocMaxBlocks) {
    set_last_error("ehdg_trace_residual_noalloc: internal block count exceeds the scratch");
    return EHDG_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(std::string("ehdg_trace_residual_noalloc: device scratch lookup failed: ") +
                   cudaGetErrorString(e));
    return EHDG_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* partials = static_cast<double*>(base);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(base) +
                                                         sizeof(double) * kNoAllocMaxBlocks);
  // the array keeps the previous call's contents: the ticket must start at 0
  e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = launch_wdiff_norm(a, b, w, n, partials, ticket, out, s);
  if (e != cudaSuccess) {
    set_last_error(std::string("ehdg_trace_residual_noalloc: ") + cudaGetErrorString(e));
    return EHDG_ERR_CUDA;
  }
  return EHDG_OK;
}
