// Sum-factorised FP64 transport sweep and reconstruction for hexahedra with
// one local operator shared by every element (constant velocity, uniform
// mesh), Sec. 3 eqs. transportLocalk1 and transportLocale.
//
// The element solve is u = A^{-1} (r0 + B uhat). B only reaches the element's
// boundary nodes, and on the tensor-product element its block for face f is
// a Kronecker product (Sec. 2 spaces, Q^p on the face):
//   (B uhat)[node (a_t1, a_t2) of face f] +=
//       s_f sum_{j1, j2} TW[a_t1][j1] TW[a_t2][j2] uhat_f[j1 + q j2],
//   TW[a][j] = l_a(xi_j) om_j,  s_f = J_f |beta.n_f|
// (the face's own Gauss rule, the face Jacobian and |beta.n| of the local
// equation's face term), so it costs two 1D passes per face instead of a
// dense product. The rest, A^{-1} restricted to the boundary-node columns, is
// dense: the sweep applies Dy = Ey A^{-1}[:, bnd] (the face-point rows the
// trace formula reads) and the reconstruction Ab = A^{-1}[:, bnd]:
//   sweep:           Y = Gy + Dy (Bs uhat)        per element 2 nb q^3 + rows nb FMAs
//   reconstruction:  u = G + Ab (Bs uhat)         2 nb q^3 + n nb
// At p = 3 (q = 4, 56 boundary nodes, 48 upwind rows) the sweep's products
// drop from 48 x 96 = 4,608 to 768 + 2,688 = 3,456 FMAs per element, and the
// reconstruction's from 64 x 96 = 6,144 to 768 + 3,584 = 4,352. The FP64 pipe
// bounds both kernels, so the time follows the FMA count.
//
// The second pass runs per boundary node over the faces that contain it, in
// face order, so the sum over faces is formed by one thread in a fixed order
// (deterministic, no atomics). Owner writes of the trace, the residual and the
// mixed-precision residual output are those of the fused sweep.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "ehdg_internal.h"
#include "sweep_common.cuh"

namespace ehdg {

namespace {

constexpr int kSfMaxBlocks = 4096;
constexpr int kSfMaxNB = 56;          // boundary nodes of a p = 3 hexahedron

struct SfParams {
  int64_t nel, nface;
  int n_rows, n_up;
  const int* rows;              // [n_rows] face-point slot of each row, upwind first
  const int32_t* elem_face;     // [6][nel]
  const double* face_jf;        // [nface]
  double fw[kMaxQ * kMaxQ];     // face Gauss weight of each face point
  double tw[kMaxP1 * kMaxQ];    // TW[a * q + j] = l_a(xi_j) om_j
  double s[6];                  // J_f |beta.n_f| of each local face
  int bmap[kSfMaxNB * 3];       // per boundary node: f | a_t1 << 4 | a_t2 << 8, or -1
  const double* Dy;             // [NQFS][NB] rows at every face point
  const double* Ab;             // [n][NB]
  // sweep
  double* uhat;                 // [2][Nqf][nface]
  IterState* it;
  const double* Gy;             // [slot][nel]
  double* Y;                    // tangential rows, for the finishing kernel
  float* R_out;                 // mixed precision: F(uhat) - uhat at owned points (or null)
  double* partials;
  int final_here;
  double tol, res_scale;
  int max_iter;
  double* hist;
  int graph_mode;
  cudaGraphConditionalHandle handle;
  // reconstruction
  int n, cn;
  const double* G;
  double* u;
};

// Bs uhat of the tile's elements: uh [NQ][32] (face points) -> [NB][32]
// (boundary nodes) in tmp, through tmp [NQ][32] itself: the second pass keeps
// its results in registers until every thread has read the first pass's.
// Threads t = 0 .. FT-1 of each lane.
template <int P1, int FT>
__device__ __forceinline__ void sf_face_passes(const SfParams& p, const double* uh, double* tmp,
                                               int lane, int t) {
  constexpr int NQF = P1 * P1, NQ = 6 * NQF;
  constexpr int NB = P1 * P1 * P1 - (P1 - 2) * (P1 - 2) * (P1 - 2);
  // pass 1: tmp[f][j2][a1] = sum_j1 TW[a1][j1] uhat_f[j1 + q j2]
  for (int o = t; o < NQ; o += FT) {
    const int f = o / NQF, rem = o - f * NQF, j2 = rem / P1, a1 = rem - j2 * P1;
    const double* u = uh + (f * NQF + j2 * P1) * 32 + lane;
    const double* w = p.tw + a1 * P1;
    double v = 0.0;
#pragma unroll
    for (int j1 = 0; j1 < P1; ++j1) v = fma(w[j1], u[j1 * 32], v);
    tmp[o * 32 + lane] = v;
  }
  __syncthreads();
  // pass 2: rb[b] = sum over the faces f of node b of
  //         s_f sum_j2 TW[a_t2][j2] tmp[f][j2][a_t1]
  constexpr int NBT = (NB + FT - 1) / FT;
  double rv[NBT];
#pragma unroll
  for (int k = 0; k < NBT; ++k) {
    const int b = t + k * FT;
    double v = 0.0;
    if (b < NB) {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int e = p.bmap[b * 3 + m];
        if (e < 0) break;
        const int f = e & 15, a1 = (e >> 4) & 15, a2 = (e >> 8) & 15;
        const double* w = p.tw + a2 * P1;
        const double* u = tmp + (f * NQF + a1) * 32 + lane;
        double x = 0.0;
#pragma unroll
        for (int j2 = 0; j2 < P1; ++j2) x = fma(w[j2], u[j2 * P1 * 32], x);
        v = fma(p.s[f], x, v);
      }
    }
    rv[k] = v;
  }
  __syncthreads();                                    // every thread done reading pass 1
#pragma unroll
  for (int k = 0; k < NBT; ++k) {
    const int b = t + k * FT;
    if (b < NB) tmp[b * 32 + lane] = rv[k];
  }
}

template <int P1, int FT>
__global__ void __launch_bounds__(32 * FT) k_sweep_sf(const SfParams p) {
  constexpr int NQF = P1 * P1, NQ = 6 * NQF;
  constexpr int NB = P1 * P1 * P1 - (P1 - 2) * (P1 - 2) * (P1 - 2);
  extern __shared__ double sm[];
  const int lane = threadIdx.x, t = threadIdx.y;
  double* Dsh = sm;                                   // [n_rows][NB]
  double* uh = Dsh + p.n_rows * NB;                   // [NQ][32]
  double* tmp = uh + NQ * 32;                         // [NQ][32], then [NB][32] boundary values
  const double* rb = tmp;
  int* fid = reinterpret_cast<int*>(tmp + NQ * 32);   // [6][32]
  for (int i = t * 32 + lane; i < p.n_rows * NB; i += 32 * FT) {
    const int j = i / NB, b = i - j * NB;
    Dsh[i] = p.Dy[p.rows[j] * NB + b];
  }
  const int64_t ne = p.nel, nface = p.nface;
  const int kk = p.it->k;                             // read before the last block advances it
  const int64_t tlen = (int64_t)NQF * nface;
  const double* src = p.uhat + (int64_t)(kk & 1) * tlen;
  double* dst = p.uhat + (int64_t)((kk + 1) & 1) * tlen;
  const int64_t ntiles = (ne + 31) / 32;
  double acc_res = 0.0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e = tile * 32 + lane;
    const bool live = e < ne;
    __syncthreads();                                  // previous tile done with smem
    if (live)
      for (int f = t; f < 6; f += FT) fid[f * 32 + lane] = p.elem_face[f * ne + e];
    __syncthreads();
    for (int i = t; i < NQ; i += FT) {
      const int f = i / NQF, g = i - f * NQF;
      uh[i * 32 + lane] = live ? src[g * nface + fid[f * 32 + lane]] : 0.0;
    }
    __syncthreads();
    sf_face_passes<P1, FT>(p, uh, tmp, lane, t);
    __syncthreads();
    if (!live) continue;
    for (int j = t; j < p.n_rows; j += FT) {
      const double* D = Dsh + j * NB;
      double a0 = p.Gy[j * ne + e], a1 = 0.0;
#pragma unroll
      for (int b = 0; b < NB; b += 2) {
        a0 = fma(D[b], rb[b * 32 + lane], a0);
        a1 = fma(D[b + 1], rb[(b + 1) * 32 + lane], a1);
      }
      const double acc = a0 + a1;
      const int r = p.rows[j];
      if (j < p.n_up) {
        const int f = r / NQF, g = r - f * NQF;
        const int face = fid[f * 32 + lane];
        dst[g * nface + face] = acc;
        const double d = acc - uh[r * 32 + lane];
        acc_res += p.face_jf[face] * p.fw[g] * d * d;
        if (p.R_out) p.R_out[g * nface + face] = (float)d;
      } else {
        p.Y[(int64_t)r * ne + e] = acc;
      }
    }
  }
  if (p.final_here) {
    finish_residual(acc_res, p.partials, blockIdx.x, gridDim.x, p.it, p.hist, p.max_iter, p.tol,
                    p.res_scale, p.graph_mode, p.handle, gridDim.x);
  } else {
    // partial sums only; the finishing kernel of tangential points reduces them
    acc_res = fsum_warp(acc_res);
    __shared__ double red2[32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) red2[tid >> 5] = acc_res;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)((blockDim.x * blockDim.y) >> 5); ++w) s += red2[w];
      p.partials[blockIdx.x] = s;
    }
  }
}

// u^{k+1} = G + Ab (Bs uhat^k) (Crank-Nicolson: 2 v - u^n), with uhat^k the
// trace the last sweep read.
template <int P1, int FT>
__global__ void __launch_bounds__(32 * FT) k_final_sf(const SfParams p) {
  constexpr int NQF = P1 * P1, NQ = 6 * NQF;
  constexpr int NB = P1 * P1 * P1 - (P1 - 2) * (P1 - 2) * (P1 - 2);
  extern __shared__ double sm[];
  const int lane = threadIdx.x, t = threadIdx.y;
  double* Ash = sm;                                   // [n][NB]
  double* uh = Ash + p.n * NB;
  double* tmp = uh + NQ * 32;
  const double* rb = tmp;
  for (int i = t * 32 + lane; i < p.n * NB; i += 32 * FT) Ash[i] = p.Ab[i];
  const int64_t ne = p.nel, nface = p.nface;
  const double* src = p.uhat + (int64_t)((p.it->k + 1) & 1) * NQF * nface;
  const int64_t ntiles = (ne + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e = tile * 32 + lane;
    const bool live = e < ne;
    __syncthreads();
    for (int i = t; i < NQ; i += FT) {
      const int f = i / NQF, g = i - f * NQF;
      uh[i * 32 + lane] = live ? src[g * nface + p.elem_face[f * ne + e]] : 0.0;
    }
    __syncthreads();
    sf_face_passes<P1, FT>(p, uh, tmp, lane, t);
    __syncthreads();
    if (!live) continue;
    for (int r = t; r < p.n; r += FT) {
      const double* A = Ash + r * NB;
      double a0 = p.G[r * ne + e], a1 = 0.0;
#pragma unroll
      for (int b = 0; b < NB; b += 2) {
        a0 = fma(A[b], rb[b * 32 + lane], a0);
        a1 = fma(A[b + 1], rb[(b + 1) * 32 + lane], a1);
      }
      double acc = a0 + a1;
      if (p.cn) acc = 2.0 * acc - p.u[r * ne + e];
      p.u[r * ne + e] = acc;
    }
  }
}

SfParams sf_params(const Ctx& c) {
  SfParams p = {};
  p.nel = c.nel;
  p.nface = c.nface;
  p.n_rows = c.n_rows;
  p.n_up = c.n_up;
  p.rows = c.rows;
  p.elem_face = c.geo.elem_face;
  p.face_jf = c.geo.face_jf;
  fill_face_weights(c, p.fw);
  const int q = c.q;
  for (int a = 0; a < q; ++a)
    for (int j = 0; j < q; ++j) p.tw[a * q + j] = c.r1d.L[j * (c.p + 1) + a] * c.r1d.om[j];
  for (int f = 0; f < 6; ++f) p.s[f] = c.sf_s[f];
  for (int i = 0; i < kSfMaxNB * 3; ++i) p.bmap[i] = i < (int)c.sf_map.size() ? c.sf_map[i] : -1;
  p.Dy = c.sf_Dy;
  p.Ab = c.sf_Ab;
  p.n = c.n;
  p.cn = (c.scheme == EHDG_CN) ? 1 : 0;
  return p;
}

template <class K>
int sf_grid(K kernel, int threads, size_t smem, int64_t ntiles) {
  const int bpsm = fn_blocks_per_sm((const void*)kernel, threads, smem);
  int64_t g = (int64_t)bpsm * device_sms();
  if (g > ntiles) g = ntiles;
  if (g > kSfMaxBlocks) g = kSfMaxBlocks;
  return g < 1 ? 1 : (int)g;
}

template <int P1, int FT>
cudaError_t launch_sweep_sf_t(const SfParams& p, cudaStream_t s, int* grid_out) {
  constexpr int NQ = 6 * P1 * P1;
  constexpr int NB = P1 * P1 * P1 - (P1 - 2) * (P1 - 2) * (P1 - 2);
  const size_t smem = sizeof(double) * ((size_t)p.n_rows * NB + 2 * NQ * 32) +
                      sizeof(int) * 6 * 32;
  cudaError_t err = fn_smem((const void*)k_sweep_sf<P1, FT>, smem);
  if (err != cudaSuccess) return err;
  const int grid = sf_grid(k_sweep_sf<P1, FT>, 32 * FT, smem, (p.nel + 31) / 32);
  *grid_out = grid;
  k_sweep_sf<P1, FT><<<grid, dim3(32, FT), smem, s>>>(p);
  return cudaGetLastError();
}

template <int P1>
cudaError_t launch_sweep_sf_p(const SfParams& p, int ft, cudaStream_t s, int* grid_out) {
  switch (ft) {
    case 2: return launch_sweep_sf_t<P1, 2>(p, s, grid_out);
    case 8: return launch_sweep_sf_t<P1, 8>(p, s, grid_out);
    default: return launch_sweep_sf_t<P1, 4>(p, s, grid_out);
  }
}

template <int P1>
cudaError_t launch_final_sf_t(const SfParams& p, cudaStream_t s) {
  constexpr int FT = 4;
  constexpr int NQ = 6 * P1 * P1;
  constexpr int NB = P1 * P1 * P1 - (P1 - 2) * (P1 - 2) * (P1 - 2);
  const size_t smem = sizeof(double) * ((size_t)p.n * NB + 2 * NQ * 32);
  cudaError_t err = fn_smem((const void*)k_final_sf<P1, FT>, smem);
  if (err != cudaSuccess) return err;
  const int grid = sf_grid(k_final_sf<P1, FT>, 32 * FT, smem, (p.nel + 31) / 32);
  k_final_sf<P1, FT><<<grid, dim3(32, FT), smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

bool sf_supported(const Ctx& c) {
  return c.pde == EHDG_TRANSPORT && c.shared_op && c.dim == 3 && !c.variable_beta &&
         c.q == c.p + 1 && c.p >= 1 && c.p <= 3;
}

// Boundary nodes, the faces of each (with the node's tangential GLL indices on
// that face), s_f, and the device arrays the assembly fills (Ab, Dy).
ehdg_status sf_prepare(Ctx& c) {
  const int P1 = c.p + 1;
  std::vector<int> bnd;
  c.sf_map.clear();
  for (int i = 0; i < c.Np; ++i) {
    const int a[3] = {i % P1, (i / P1) % P1, i / (P1 * P1)};
    std::vector<int> ent;
    for (int f = 0; f < 6; ++f) {
      const int ax = f >> 1, side = f & 1;
      if (a[ax] != (side ? P1 - 1 : 0)) continue;
      int t[2], k = 0;
      for (int d = 0; d < 3; ++d)
        if (d != ax) t[k++] = a[d];
      ent.push_back(f | (t[0] << 4) | (t[1] << 8));
    }
    if (ent.empty()) continue;
    bnd.push_back(i);
    for (int m = 0; m < 3; ++m) c.sf_map.push_back(m < (int)ent.size() ? ent[m] : -1);
  }
  c.sf_NB = (int)bnd.size();
  if (c.sf_NB > kSfMaxNB) return EHDG_ERR_UNSUPPORTED;
  // J_f |beta.n_f| (uniform mesh: one element's edge lengths serve all)
  for (int f = 0; f < 6; ++f) {
    const int ax = f >> 1;
    double jf = 1.0;
    for (int d = 0; d < 3; ++d)
      if (d != ax) jf *= 0.5 * c.elem_h[d];
    c.sf_s[f] = jf * std::fabs(c.beta_const[ax]);
  }
  if (dalloc_raw(c, (void**)&c.sf_bnd, sizeof(int) * bnd.size()) != cudaSuccess ||
      dalloc_raw(c, (void**)&c.sf_Ab, sizeof(double) * c.n * c.sf_NB) != cudaSuccess ||
      dalloc_raw(c, (void**)&c.sf_Dy, sizeof(double) * c.NQFS * c.sf_NB) != cudaSuccess) {
    cudaGetLastError();
    return EHDG_ERR_OOM;
  }
  if (cudaMemcpy(c.sf_bnd, bnd.data(), sizeof(int) * bnd.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return EHDG_ERR_CUDA;
  return EHDG_OK;
}

cudaError_t launch_sweep_sf(Ctx& c, int graph_mode, int* grid_out) {
  SfParams p = sf_params(c);
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
  switch (c.p + 1) {
    case 2: return launch_sweep_sf_p<2>(p, c.sweep_ft, c.stream, grid_out);
    case 3: return launch_sweep_sf_p<3>(p, c.sweep_ft, c.stream, grid_out);
    default: return launch_sweep_sf_p<4>(p, c.sweep_ft, c.stream, grid_out);
  }
}

cudaError_t launch_final_sf(Ctx& c) {
  SfParams p = sf_params(c);
  p.uhat = c.uhat;
  p.it = c.it;
  p.G = c.G;
  p.u = c.u;
  switch (c.p + 1) {
    case 2: return launch_final_sf_t<2>(p, c.stream);
    case 3: return launch_final_sf_t<3>(p, c.stream);
    default: return launch_final_sf_t<4>(p, c.stream);
  }
}

}  // namespace ehdg
