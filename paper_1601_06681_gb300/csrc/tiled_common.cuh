// Shared pieces of the tiled per-element kernels (sweep, correction sweep,
// reconstruction): launch constants, bulk-copy issue and bounded mbarrier
// waits, and the launch shape. Every wait gives up after a bounded number of
// polls, so no kernel built on these can hang on a copy that never lands.
#pragma once

#include <cuda_runtime.h>

#include "ehdg_internal.h"

namespace ehdg {

namespace {

// compile-time tuning: warps per block (independent of each other), stages
// per warp, independent FMA chains per row
#ifndef EHDG_TILED_TW
#define EHDG_TILED_TW 4
#endif
#ifndef EHDG_TILED_TS
#define EHDG_TILED_TS 2
#endif
#ifndef EHDG_TILED_CH
#define EHDG_TILED_CH 1
#endif
// minimum resident blocks per SM asked of the compiler (instances with up
// to 28 face points per element)
#ifndef EHDG_TILED_MINB
#define EHDG_TILED_MINB 3
#endif
constexpr int kTW = EHDG_TILED_TW;
constexpr int kTS = EHDG_TILED_TS;
constexpr int kCH = EHDG_TILED_CH;
static_assert(kCH == 1 || kCH == 2 || kCH == 4, "FMA chains per row: 1, 2 or 4");
constexpr uint32_t kTileWaitLimit = 1u << 22; // mbarrier polls before giving up
constexpr uint32_t kBarrierPolls = 1u << 22;  // grid-barrier polls before giving up
constexpr int kTiledMaxBlocks = 4096;         // same bound as the other transport sweep

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// lane 0 only: start the copy of one operator row into a stage
__device__ __forceinline__ void issue_row(uint32_t mbar, uint32_t dst, const void* src,
                                          uint32_t bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// bounded wait for a phase of an mbarrier; true when it completed
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity,
                                           uint32_t limit = kTileWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
        " selp.u32 %0, 1, 0, w;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// bounded wait polled by every lane of a warp (each lane then sees the
// stage's data); the result is warp-uniform
__device__ __forceinline__ bool wait_phase_warp(uint32_t mbar, uint32_t parity,
                                                uint32_t limit = kTileWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
        " selp.u32 %0, 1, 0, w;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (__all_sync(0xffffffffu, done)) return true;
  }
  return false;
}

// Grid-wide barrier of a cooperative launch: generation target = number of
// arrivals expected so far. Thread 0 of each block arrives and polls with a
// bounded number of polls; a block that gives up, or sees another block give
// up, raises *abort. Returns the block-uniform outcome.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int target, int* abort,
                                             uint32_t polls = kBarrierPolls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 0;
    for (uint32_t it = 0; it < polls; ++it) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) {
        ok = 1;
        break;
      }
      if (*reinterpret_cast<volatile int*>(abort)) break;
      __nanosleep(32);
    }
    // an abort raised before any block arrived is seen by every block here
    if (ok && *reinterpret_cast<volatile int*>(abort)) ok = 0;
    if (!ok) atomicExch(abort, 1);
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// launch shape of one kernel instance: dynamic shared memory and a one-wave
// grid with at least four rows per warp
template <class K>
cudaError_t tiled_shape_of(K kern, int NQ, int64_t total_rows, int64_t ntiles, int* grid,
                           size_t* smem_out, size_t stage_bytes_per_value = sizeof(double) * kTS) {
  const size_t smem = stage_bytes_per_value * (size_t)kTW * NQ * 32;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  int bpsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, kern, 32 * kTW, smem) != cudaSuccess ||
      bpsm < 1) {
    cudaGetLastError();
    bpsm = 1;
  }
  int64_t g = (int64_t)bpsm * device_sms();
  const int64_t by_rows = (total_rows + 4 * kTW - 1) / (4 * kTW);
  if (g > by_rows) g = by_rows;
  if (g > ntiles) g = ntiles;
  if (g > kTiledMaxBlocks) g = kTiledMaxBlocks;
  if (g < 1) g = 1;
  *grid = (int)g;
  *smem_out = smem;
  return cudaSuccess;
}

}  // namespace

}  // namespace ehdg

// (faces, points per face) pairs with an instance of the tiled kernels:
// quadrilaterals with 2..10 Gauss points per edge, hexahedra with 2x2 or 3x3
// per face
#define EHDG_TILED_SHAPES(X) \
  X(4, 2) X(4, 3) X(4, 4) X(4, 5) X(4, 6) X(4, 7) X(4, 8) X(4, 9) X(4, 10) X(6, 4) X(6, 9)
