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

}  // namespace

}  // namespace ehdg

extern "C" ehdg_status ehdg_selftest_wait_timeout(int which, void* stream) {
  using namespace ehdg;
  if (which != 0 && which != 1) {
    set_last_error("ehdg_selftest_wait_timeout: which must be 0 (mbarrier) or 1 (grid barrier)");
    return EHDG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
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
