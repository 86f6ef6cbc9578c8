// Transport sweep for per-element operators (variable velocity), with the
// operator streamed into shared memory by bulk asynchronous copies
// (Sec. 3: eq. transportLocalk1 with the element solve folded into Hy, then
// the trace formula eq. transportLocale).
//
// The operator rows are kept a second time in a tile-major layout: for each
// tile of 32 elements, the rows (slots) any of its elements needs, each row
// NQFS columns x 32 elements of FP64 (7 KB for NQFS = 28), contiguous, the
// tiles one after the other. Every warp takes an equal contiguous range of
// these rows and streams it through a ring of kTS shared-memory stages with
// cp.async.bulk, one mbarrier per stage, so the copies of its next rows are in
// flight while the FMAs of the current row run. A lane is an element: its
// trace values, face ids and face Jacobians are gathered into registers when
// the warp enters a tile.
//
// The trace update follows the same owner-writes rule as the other transport
// sweep: the upwind element writes uhat^{k+1} at its outflow points and adds
// the point's share of ||uhat^{k+1} - uhat^k||^2; rows of points with
// beta.n = 0 go to Y for the finishing kernel.
//
// Every mbarrier wait is bounded; a wait that gives up sets *err, and the
// block waits (bounded again) for its copies still in flight before it ends.
#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "sweep_common.cuh"
#include "tiled_common.cuh"
#include "sweep_pass.cuh"

namespace ehdg {

namespace {

// One eHDG iteration per launch; the last block to finish reduces the
// residual and sets the loop condition of the step's graph.
template <int F, int NQF>
__global__ void __launch_bounds__(32 * kTW, (F * NQF <= 28) ? EHDG_TILED_MINB : 1)
    k_sweep_tiled(const TiledParams p) {
  constexpr int NQ = F * NQF;
  extern __shared__ __align__(256) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar[kTW][kTS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* stages = reinterpret_cast<double*>(tsm) + (size_t)w * kTS * NQ * 32;
  const uint32_t mbar0 = saddr(&mbar[w][0]);
  const int kk = p.it->k;                        // read before the last block advances it
  const int64_t tlen = (int64_t)NQF * p.nface;
  const double* src = p.uhat + (int64_t)(kk & 1) * tlen;
  double* dst = p.uhat + (int64_t)((kk + 1) & 1) * tlen;
  const int64_t nwarps = (int64_t)gridDim.x * kTW, gw = (int64_t)blockIdx.x * kTW + w;
  const int64_t J0 = p.total_rows * gw / nwarps, J1 = p.total_rows * (gw + 1) / nwarps;
  int64_t qp = 0, q_done = 0;
  ring_init(mbar0, kTS, lane);
  ring_fill(p.Hyt, stages, mbar0, kTS, NQ, lane, J0, J1 - J0, 0, qp, J1 - J0);
  double acc_res = 0.0;
  sweep_pass<F, NQF, false>(p, stages, mbar0, lane, gw, J0, J1, 0, q_done, qp, J1 - J0, src, dst,
                            acc_res);
  ring_drain(mbar0, kTS, lane, q_done, qp);
  if (p.final_here) {
    finish_residual(acc_res, p.partials, blockIdx.x, gridDim.x, p.it, p.hist, p.max_iter, p.tol,
                    p.res_scale, p.graph_mode, p.handle, gridDim.x);
  } else {
    __shared__ double red[kTW];
    const double v = fsum_warp(acc_res);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < kTW; ++i) s += red[i];
      p.partials[blockIdx.x] = s;
    }
  }
}

// All iterations of one implicit step in one cooperative launch (every block
// resident): pass k reads uhat^k from slot k & 1 and writes uhat^{k+1} to the
// other slot; after a grid barrier every block sums the blocks' residual
// partials in the same order, so every block takes the same decision (the
// rule of the per-iteration kernel: stop when r_k < tol, when r_k is not
// finite, or after max_iter iterations). The warps keep streaming their rows
// across passes, so the first rows of the next pass arrive during the
// barrier. Block 0 records the history and the final iteration state.
template <int F, int NQF>
__global__ void __launch_bounds__(32 * kTW, (F * NQF <= 28) ? EHDG_TILED_MINB : 1)
    k_sweep_persist(const TiledParams p) {
  constexpr int NQ = F * NQF;
  extern __shared__ __align__(256) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar[kTW][kTS];
  __shared__ double red[kTW];
  __shared__ double s_r;
  __shared__ int s_cont, s_status;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* stages = reinterpret_cast<double*>(tsm) + (size_t)w * kTS * NQ * 32;
  const uint32_t mbar0 = saddr(&mbar[w][0]);
  const int k0 = p.it->k;
  const int64_t tlen = (int64_t)NQF * p.nface;
  const int64_t nwarps = (int64_t)gridDim.x * kTW, gw = (int64_t)blockIdx.x * kTW + w;
  const int64_t J0 = p.total_rows * gw / nwarps, J1 = p.total_rows * (gw + 1) / nwarps;
  const int64_t L = J1 - J0;
  const int passes = p.max_iter - k0 > 0 ? p.max_iter - k0 : 1;
  int64_t qp = 0, q_done = 0;
  ring_init(mbar0, kTS, lane);
  ring_fill(p.Hyt, stages, mbar0, kTS, NQ, lane, J0, L, 0, qp, L * passes);
  int k = k0;
  bool ok = true;
  for (int pass = 0; pass < passes; ++pass) {
    const double* src = p.uhat + (int64_t)(k & 1) * tlen;
    double* dst = p.uhat + (int64_t)((k + 1) & 1) * tlen;
    double acc_res = 0.0;
    if (!sweep_pass<F, NQF, true>(p, stages, mbar0, lane, gw, J0, J1, (int64_t)pass * L, q_done,
                                  qp, L * passes, src, dst, acc_res))
      atomicExch(&p.it->abort, 1);
    const double v = fsum_warp(acc_res);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < kTW; ++i) s += red[i];
      p.partials[(int64_t)(pass & 1) * gridDim.x + blockIdx.x] = s;
    }
    if (!grid_barrier(&p.it->bar, (unsigned int)(pass + 1) * gridDim.x, &p.it->abort)) {
      ok = false;
      break;
    }
    // the residual of this pass, summed by warp 0 in a fixed order
    if (w == 0) {
      const double* part = p.partials + (int64_t)(pass & 1) * gridDim.x;
      double s = 0.0;
      for (int i = lane; i < (int)gridDim.x; i += 32) s += __ldcg(part + i);
      s = fsum_warp(s);
      if (lane == 0) {
        const double r = p.res_scale * sqrt(s);
        int cont = 1, status = EHDG_OK;
        if (!isfinite(r)) { cont = 0; status = EHDG_ERR_DIVERGED; }
        else if (r < p.tol) { cont = 0; status = EHDG_OK; }
        else if (k + 1 >= p.max_iter) { cont = 0; status = EHDG_ERR_NOT_CONVERGED; }
        s_r = r;
        s_cont = cont;
        s_status = status;
        if (blockIdx.x == 0 && k < p.max_iter) p.hist[k] = r;
      }
    }
    __syncthreads();
    ++k;
    if (!s_cont) break;
  }
  ring_drain(mbar0, kTS, lane, q_done, qp);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.it->k = k;
    p.it->r_last = ok ? s_r : p.it->r_last;
    p.it->cont = 0;
    p.it->status = ok ? s_status : EHDG_ERR_TIMEOUT;
    __threadfence();
  }
}

template <int F, int NQF>
cudaError_t tiled_config(int64_t total_rows, int64_t ntiles, int* grid, size_t* smem_out) {
  return tiled_shape_of(k_sweep_tiled<F, NQF>, F * NQF, total_rows, ntiles, grid, smem_out);
}

template <int F, int NQF>
cudaError_t tiled_launch(const TiledParams& p, int grid, size_t smem, cudaStream_t s) {
  k_sweep_tiled<F, NQF><<<grid, 32 * kTW, smem, s>>>(p);
  return cudaGetLastError();
}

// blocks of the persistent kernel that fit on one SM (0 on error)
template <int F, int NQF>
int persist_blocks_per_sm(size_t smem) {
  auto kern = k_sweep_persist<F, NQF>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int bpsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, kern, 32 * kTW, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return bpsm;
}

template <int F, int NQF>
cudaError_t persist_launch(const TiledParams& p, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<TiledParams*>(&p)};
  return cudaLaunchCooperativeKernel((const void*)k_sweep_persist<F, NQF>, dim3(grid),
                                     dim3(32 * kTW), args, smem, s);
}

struct SweepOps {
  cudaError_t (*config)(int64_t, int64_t, int*, size_t*);
  cudaError_t (*launch)(const TiledParams&, int, size_t, cudaStream_t);
  int (*persist_bpsm)(size_t);
  cudaError_t (*persist)(const TiledParams&, int, size_t, cudaStream_t);
};

bool sweep_ops(int F, int Nqf, SweepOps* out) {
#define EHDG_SWEEP_CASE(f_, q_)                                     \
  if (F == f_ && Nqf == q_) {                                       \
    *out = SweepOps{&tiled_config<f_, q_>, &tiled_launch<f_, q_>,   \
                    &persist_blocks_per_sm<f_, q_>, &persist_launch<f_, q_>}; \
    return true;                                                    \
  }
  EHDG_TILED_SHAPES(EHDG_SWEEP_CASE)
#undef EHDG_SWEEP_CASE
  return false;
}

}  // namespace

bool tiled_supported(const Ctx& c) {
  SweepOps ops;
  return c.pde == EHDG_TRANSPORT && !c.shared_op && sweep_ops(c.F, c.Nqf, &ops);
}

cudaError_t tiled_sweep_shape(const Ctx& c, int64_t rows, int64_t ntiles, int* grid,
                              size_t* smem) {
  SweepOps ops;
  if (!sweep_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  return ops.config(rows, ntiles, grid, smem);
}

static void fill_params(Ctx& c, TiledParams& p, int graph_mode) {
  p.nel = c.nel;
  p.nface = c.nface;
  p.ntiles = c.ntiles;
  p.total_rows = c.tile_rows;
  p.warp_tile = c.tiled_warp_tile;
  p.rowid = c.rowid;
  p.nrows = c.nrows;
  p.nup = c.nup;
  p.elem_face = c.geo.elem_face;
  p.face_jf = c.geo.face_jf;
  fill_face_weights(c, p.fw);
  p.Hyt = c.Hyt;
  p.tile_row0 = c.tile_row0;
  p.tile_nrows = c.tile_nrows;
  p.uhat = c.uhat;
  p.it = c.it;
  p.Gy = c.Gy;
  p.Y = c.Y;
  p.R_out = c.mixed ? c.R32 : nullptr;
  p.partials = c.partials;
  p.final_here = c.n_tan == 0 ? 1 : 0;
  p.tol = c.tol;
  p.res_scale = c.res_scale;
  p.max_iter = c.max_iter;
  p.hist = c.hist;
  p.graph_mode = graph_mode;
  p.handle = c.handle;
  p.err = c.tc_err;
}

cudaError_t launch_sweep_tiled(Ctx& c, int graph_mode, int* grid_out) {
  TiledParams p;
  fill_params(c, p, graph_mode);
  SweepOps ops;
  if (!sweep_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  *grid_out = c.tiled_grid;
  return ops.launch(p, c.tiled_grid, c.tiled_smem, c.stream);
}

int tiled_persist_blocks_per_sm(const Ctx& c) {
  SweepOps ops;
  if (!sweep_ops(c.F, c.Nqf, &ops)) return 0;
  return ops.persist_bpsm(c.tiled_smem);
}

bool persistent_sweep_ok(const Ctx& c) {
  return c.Hyt && c.persist_fits && c.ppartials && !c.mixed && c.n_tan == 0;
}

cudaError_t launch_sweep_persistent(Ctx& c) {
  TiledParams p;
  fill_params(c, p, 0);
  p.partials = c.ppartials;
  SweepOps ops;
  if (!sweep_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  return ops.persist(p, c.tiled_grid, c.tiled_smem, c.stream);
}

}  // namespace ehdg
