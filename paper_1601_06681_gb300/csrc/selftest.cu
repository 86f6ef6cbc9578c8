// Self-test of the bounded device-side waits used by the tiled and persistent
// sweeps. Each case runs the wait those kernels use against a condition that
// nothing will ever satisfy, with a short poll limit: the wait must give up,
// the kernel must report it through a flag that the host reads, and the
// device must stay usable afterwards. No case faults, traps or hangs: every
// loop below is bounded.
#include <cuda_runtime.h>

#include <string>

#include "ehdg_internal.h"
#include "tiled_common.cuh"

namespace ehdg {

namespace {

constexpr uint32_t kSelftestPolls = 4096;
constexpr int kProbeChains = 8;        // independent FMA chains per thread
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 4;

// written only when a chain ends on a value it cannot reach, so the chains
// stay live without any store in practice
__device__ double g_probe_sink;

// An mbarrier that expects one arrival; none ever comes, so phase 0 never
// completes. Both the warp-wide and the single-thread wait must give up.
__global__ void k_wait_never_mbarrier(int* flag) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t a = saddr(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool warp_done = wait_phase_warp(a, 0u, kSelftestPolls);
  const bool one_done = (threadIdx.x == 0) ? wait_phase(a, 0u, kSelftestPolls) : true;
  if (threadIdx.x == 0 && !warp_done && !one_done) atomicAdd(flag, 1);
}

// A grid barrier whose target counts one more arrival than the grid has
// blocks: every block must give up and raise the abort flag.
__global__ void k_wait_never_barrier(unsigned int* bar, int* abort, int* flag) {
  const bool done = grid_barrier(bar, gridDim.x + 1u, abort, kSelftestPolls);
  if (threadIdx.x == 0 && !done) atomicAdd(flag, 1);
}

// n_iter steps of kProbeChains independent FP64 FMA chains per thread: the
// chains hide the FMA latency, so the FP64 pipe runs at its issue rate.
__global__ void __launch_bounds__(kProbeThreads) k_dfma_chains(int n_iter, double b, double c) {
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0 + 1e-3 * k + 1e-9 * threadIdx.x;
#pragma unroll 4
  for (int i = 0; i < n_iter; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == -1.0) g_probe_sink = s;
}

}  // namespace

}  // namespace ehdg

extern "C" ehdg_status ehdg_probe_fp64_rate(void* stream, int* sms, double* tflops) {
  using namespace ehdg;
  if (!tflops) {
    set_last_error("ehdg_probe_fp64_rate: tflops is NULL");
    return EHDG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n_sm = device_sms();
  const int blocks = n_sm * kProbeBlocksPerSM;
  constexpr int kIter = 1 << 14;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best_ms = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms up
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess) {
      k_dfma_chains<<<blocks, kProbeThreads, 0, s>>>(kIter, 0.999999999, 1e-12);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess || !(best_ms > 0.f)) {
    cudaGetLastError();
    set_last_error(std::string("ehdg_probe_fp64_rate: ") +
                   (e != cudaSuccess ? cudaGetErrorString(e) : "no timing"));
    return EHDG_ERR_CUDA;
  }
  const double flops = 2.0 * kProbeChains * (double)kIter * blocks * kProbeThreads;
  *tflops = flops / (best_ms * 1e-3) / 1e12;
  if (sms) *sms = n_sm;
  return EHDG_OK;
}

extern "C" ehdg_status ehdg_selftest_wait_timeout(int which, void* stream) {
  using namespace ehdg;
  if (which < 0 || which > 2) {
    set_last_error("ehdg_selftest_wait_timeout: which must be 0 (mbarrier), 1 (grid barrier) or "
                   "2 (work ring)");
    return EHDG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (which == 2) {
    int gave_up = 0;
    const cudaError_t er = batch_ring_selftest(s, 1u << 12, &gave_up);
    if (er != cudaSuccess) {
      cudaGetLastError();
      set_last_error(std::string("ehdg_selftest_wait_timeout: ") + cudaGetErrorString(er));
      return EHDG_ERR_CUDA;
    }
    if (!gave_up) {
      set_last_error("ehdg_selftest_wait_timeout: the work ring's wait did not give up");
      return EHDG_OK;
    }
    set_last_error("ehdg_selftest_wait_timeout: every bounded wait gave up, as designed");
    return EHDG_ERR_TIMEOUT;
  }
  constexpr int kBlocks = 4;
  int* buf = nullptr;              // [0] barrier count, [1] abort, [2] gave-up count
  cudaError_t e = cudaMallocAsync((void**)&buf, 4 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 4 * sizeof(int), s);
  int expected = 1;
  if (e == cudaSuccess) {
    if (which == 0) {
      k_wait_never_mbarrier<<<1, 32, 0, s>>>(buf + 2);
    } else {
      k_wait_never_barrier<<<kBlocks, 64, 0, s>>>(reinterpret_cast<unsigned int*>(buf), buf + 1,
                                                   buf + 2);
      expected = kBlocks;
    }
    e = cudaGetLastError();
  }
  int gave_up = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&gave_up, buf + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (buf) cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(std::string("ehdg_selftest_wait_timeout: ") + cudaGetErrorString(e));
    return EHDG_ERR_CUDA;
  }
  if (gave_up != expected) {
    set_last_error("ehdg_selftest_wait_timeout: a wait on a condition that never holds did not "
                   "give up (" + std::to_string(gave_up) + " of " + std::to_string(expected) +
                   ")");
    return EHDG_OK;
  }
  set_last_error("ehdg_selftest_wait_timeout: every bounded wait gave up, as designed");
  return EHDG_ERR_TIMEOUT;
}
