// Standalone FP64 trace residual (the convergence check of Algorithm 1):
//   r = sqrt( sum_i w_i (a_i - b_i)^2 )
// over caller-owned device arrays. Deterministic: a fixed grid of block
// partial sums, reduced in block order by the last block to finish.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "ehdg_internal.h"

namespace ehdg {

namespace {

constexpr int kResidBlock = 256;

__device__ __forceinline__ double rsum_warp(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partials[gridDim.x] and *counter are scratch; *counter must be 0 on entry
// and is 0 again on exit.
__global__ void __launch_bounds__(kResidBlock)
k_wdiff_norm(const double* __restrict__ a, const double* __restrict__ b,
             const double* __restrict__ w, int64_t n, double* partials, unsigned int* counter,
             double* out) {
  __shared__ double red[kResidBlock / 32];
  __shared__ bool last;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = a[i] - b[i];
    acc += w[i] * d * d;
  }
  acc = rsum_warp(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    v = rsum_warp(v);
    if (lane == 0) {
      partials[blockIdx.x] = v;
      __threadfence();
      last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
    v += reinterpret_cast<volatile double*>(partials)[i];
  v = rsum_warp(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    *out = sqrt(s);
    *counter = 0u;
  }
}

int resid_blocks(int64_t n) {
  int64_t b = (n + kResidBlock - 1) / kResidBlock;
  if (b > kResidMaxBlocks) b = kResidMaxBlocks;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_wdiff_norm(const double* a, const double* b, const double* w, int64_t n,
                              double* partials, unsigned int* counter, double* out,
                              cudaStream_t s) {
  k_wdiff_norm<<<resid_blocks(n), kResidBlock, 0, s>>>(a, b, w, n, partials, counter, out);
  return cudaGetLastError();
}

int wdiff_norm_blocks(int64_t n) { return resid_blocks(n); }

}  // namespace ehdg

extern "C" ehdg_status ehdg_trace_residual(const double* a, const double* b, const double* w,
                                           int64_t n, double* out, void* stream) {
  using namespace ehdg;
  if (!out || n < 0 || (n > 0 && (!a || !b || !w))) {
    set_last_error("ehdg_trace_residual: NULL pointer or negative size");
    return EHDG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = resid_blocks(n);
  void* scratch = nullptr;
  const size_t bytes = sizeof(double) * blocks + 256;
  cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error(std::string("ehdg_trace_residual: ") + cudaGetErrorString(e));
    return EHDG_ERR_OOM;
  }
  double* partials = static_cast<double*>(scratch);
  unsigned int* counter = reinterpret_cast<unsigned int*>(static_cast<char*>(scratch) +
                                                          sizeof(double) * blocks);
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = launch_wdiff_norm(a, b, w, n, partials, counter, out, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    set_last_error(std::string("ehdg_trace_residual: ") + cudaGetErrorString(e));
    return EHDG_ERR_CUDA;
  }
  return EHDG_OK;
}
