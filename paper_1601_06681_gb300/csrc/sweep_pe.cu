// FP64 transport sweep on quadrilaterals with one shared local operator, one
// thread per element (the tile body in pe_tile.cuh). Small elements (2D,
// p <= 6: 8 to 28 face points, 4 to 14 sweep rows) give a thread only a few
// hundred FMAs, so the whole element stays in registers and a tile needs no
// barrier except the residual's. Its residual reduction does not depend on
// the grid, which lets a batch iterate such instances together and still
// match their single-problem runs bit for bit.
#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "pe_tile.cuh"

namespace ehdg {

namespace {

template <int NQ>
__global__ void __launch_bounds__(kPeTile) k_sweep_pe(const __grid_constant__ PeView v,
                                                      const double* Hy, int graph_mode,
                                                      cudaGraphConditionalHandle handle) {
  __shared__ double Hsh[NQ * NQ];
  for (int i = threadIdx.x; i < v.n_rows * NQ; i += kPeTile) {
    const int j = i / NQ, c = i - j * NQ;
    Hsh[i] = Hy[v.rows[j] * NQ + c];
  }
  __syncthreads();
  const int kk = v.it->k;                     // read before the last tile advances it
  const int64_t tlen = (int64_t)(NQ / 4) * v.nface;
  const double* src = v.uhat_slot(kk & 1, tlen);
  double* dst = const_cast<double*>(v.uhat_slot((kk + 1) & 1, tlen));
  const int64_t ntiles = (v.nel + kPeTile - 1) / kPeTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    pe_tile<NQ>(v, Hsh, src, dst, tile, ntiles, graph_mode, handle);
}

template <int NQ>
cudaError_t launch_pe_t(const PeView& v, const double* Hy, int graph_mode,
                        cudaGraphConditionalHandle handle, cudaStream_t s, int* grid_out) {
  const int bpsm = fn_blocks_per_sm((const void*)k_sweep_pe<NQ>, kPeTile, 0);
  const int64_t ntiles = (v.nel + kPeTile - 1) / kPeTile;
  int64_t grid = (int64_t)bpsm * device_sms();
  if (grid > ntiles) grid = ntiles;
  *grid_out = (int)grid;
  k_sweep_pe<NQ><<<(int)grid, kPeTile, 0, s>>>(v, Hy, graph_mode, handle);
  return cudaGetLastError();
}

template <int NQ>
__global__ void __launch_bounds__(kPeTile) k_lp_pe(const LpPeView v, const float* Hy32) {
  __shared__ float Hsh[NQ * NQ];
  for (int i = threadIdx.x; i < v.n_up * NQ; i += kPeTile) {
    const int j = i / NQ, c = i - j * NQ;
    Hsh[i] = Hy32[v.rows[j] * NQ + c];
  }
  __syncthreads();
  const int64_t ntiles = (v.nel + kPeTile - 1) / kPeTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) lp_pe_tile<NQ>(v, Hsh, tile);
}

template <int NQ>
cudaError_t launch_lp_pe_t(const LpPeView& v, const float* Hy32, cudaStream_t s) {
  const int bpsm = fn_blocks_per_sm((const void*)k_lp_pe<NQ>, kPeTile, 0);
  const int64_t ntiles = (v.nel + kPeTile - 1) / kPeTile;
  int64_t grid = (int64_t)bpsm * device_sms();
  if (grid > ntiles) grid = ntiles;
  k_lp_pe<NQ><<<(int)grid, kPeTile, 0, s>>>(v, Hy32);
  return cudaGetLastError();
}

}  // namespace

// FP32 correction sweep, one thread per element (quadrilaterals, shared
// operator, no beta.n = 0 point): every sweep row is an owned point.
cudaError_t launch_lp_sweep_pe(Ctx& c, const float* in, float* out) {
  LpPeView v;
  v.nel = c.nel;
  v.nface = c.nface;
  v.n_up = c.n_up;
  v.rows = c.rows;
  v.elem_face = c.geo.elem_face;
  v.R = c.R32;
  v.in = in;
  v.out = out;
  switch (c.NQFS) {
    case 8: return launch_lp_pe_t<8>(v, c.Hy32, c.stream);
    case 12: return launch_lp_pe_t<12>(v, c.Hy32, c.stream);
    case 16: return launch_lp_pe_t<16>(v, c.Hy32, c.stream);
    case 20: return launch_lp_pe_t<20>(v, c.Hy32, c.stream);
    case 24: return launch_lp_pe_t<24>(v, c.Hy32, c.stream);
    default: return launch_lp_pe_t<28>(v, c.Hy32, c.stream);
  }
}

bool pe_supported(const Ctx& c) {
  return c.pde == EHDG_TRANSPORT && c.dim == 2 && c.shared_op && !c.variable_beta &&
         c.n_tan == 0 && !c.Hyt && c.NQFS >= 8 && c.NQFS <= 28;
}

PeView pe_view(const Ctx& c, double* fw_dev) {
  PeView v = {};
  v.nel = c.nel;
  v.nface = c.nface;
  v.n_rows = c.n_rows;
  v.n_up = c.n_up;
  v.rows = c.rows;
  v.elem_face = c.geo.elem_face;
  v.face_jf = c.geo.face_jf;
  v.fw = fw_dev;
  v.Gy = c.Gy;
  v.Y = c.Y;
  v.R_out = c.mixed ? c.R32 : nullptr;
  v.partials = c.partials;
  v.it = c.it;
  v.hist = c.hist;
  v.max_iter = c.max_iter;
  v.tol = c.tol;
  v.res_scale = c.res_scale;
  v.uhat = c.uhat;
  return v;
}

cudaError_t launch_sweep_pe(Ctx& c, int graph_mode, int* grid_out) {
  const PeView v = pe_view(c, c.pe_fw);
  switch (c.NQFS) {
    case 8: return launch_pe_t<8>(v, c.Hy, graph_mode, c.handle, c.stream, grid_out);
    case 12: return launch_pe_t<12>(v, c.Hy, graph_mode, c.handle, c.stream, grid_out);
    case 16: return launch_pe_t<16>(v, c.Hy, graph_mode, c.handle, c.stream, grid_out);
    case 20: return launch_pe_t<20>(v, c.Hy, graph_mode, c.handle, c.stream, grid_out);
    case 24: return launch_pe_t<24>(v, c.Hy, graph_mode, c.handle, c.stream, grid_out);
    default: return launch_pe_t<28>(v, c.Hy, graph_mode, c.handle, c.stream, grid_out);
  }
}

}  // namespace ehdg
