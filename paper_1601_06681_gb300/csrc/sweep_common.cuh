// Device helpers shared by the transport sweeps: warp sum and the
// deterministic last-block reduction of the trace residual (Algorithm 1,
// convergence check), which also sets the device-side loop condition.
#pragma once

#include <cuda_runtime.h>

#include "ehdg_internal.h"

namespace ehdg {

__device__ __forceinline__ double fsum_warp(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Final reduction of nblocks partials by the last block to take a ticket;
// records r_k and sets the loop condition (same rule as the trace kernel).
// partials[slot] receives this block's sum; the last of the nblocks blocks of
// this launch to take a ticket sums partials[0 .. n_total_partials).
// Returns true in the block that did the final reduction.
__device__ __forceinline__ bool finish_residual(double acc, double* partials, unsigned int slot,
                                                unsigned int nblocks, IterState* it, double* hist,
                                                int max_iter, double tol, double res_scale,
                                                int graph_mode, cudaGraphConditionalHandle handle,
                                                int n_total_partials) {
  __shared__ double red[32];
  __shared__ bool last;
  acc = fsum_warp(acc);
  const int nw = (blockDim.x * blockDim.y) >> 5;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double v = (lane < nw) ? red[lane] : 0.0;
    v = fsum_warp(v);
    if (lane == 0) {
      partials[slot] = v;
      __threadfence();
      last = (atomicAdd(&it->counter, 1u) == nblocks - 1);
    }
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double v = 0.0;
  for (int i = tid; i < n_total_partials; i += blockDim.x * blockDim.y)
    v += reinterpret_cast<volatile double*>(partials)[i];
  v = fsum_warp(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int w = 0; w < nw; ++w) sum += red[w];
    const double r = res_scale * sqrt(sum);
    const int k = it->k;
    if (k < max_iter) hist[k] = r;
    it->k = k + 1;
    it->r_last = r;
    it->counter = 0u;
    int cont = 1, status = EHDG_OK;
    if (!isfinite(r)) { cont = 0; status = EHDG_ERR_DIVERGED; }
    else if (r < tol) { cont = 0; status = EHDG_OK; }
    else if (k + 1 >= max_iter) { cont = 0; status = EHDG_ERR_NOT_CONVERGED; }
    it->cont = cont;
    it->status = status;
    __threadfence();
    if (graph_mode) cudaGraphSetConditional(handle, (unsigned int)cont);
  }
  return true;
}

}  // namespace ehdg
