// One 128-element tile of the FP64 transport sweep on quadrilaterals with one
// local operator shared by every element (Sec. 3, eqs. transportLocalk1 and
// transportLocale), one thread per element: the thread gathers its element's
// traces at its NQ face points into registers, forms every sweep row
// Y = Gy + Hy uhat (even and odd columns in two FMA chains), and as the
// upwind element writes the new trace at the points it owns, adding
// w (uhat^{k+1} - uhat^k)^2 to the residual.
//
// The residual is reduced per tile (warp sums, then the warps in order) into
// partials[tile]; the tile that takes the last ticket of the sweep adds the
// partials up in a fixed order (lane l sums tiles l, l + 32, ..., then a warp
// butterfly), records r_k and decides whether the loop goes on. The result
// depends on neither the grid nor the order in which tiles run, so the
// single-problem sweep and the batched loop, which both run this code, give
// the same iterates and residuals bit for bit.
#pragma once

#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "sweep_common.cuh"

namespace ehdg {

constexpr int kPeTile = 128;   // elements per tile = threads per block

// Loads of data that other blocks of the same launch write (traces,
// corrections, residuals): CG = true reads through L2 only (a persistent
// launch, where an SM's L1 may hold lines other SMs have rewritten since).
template <bool CG, class T>
__device__ __forceinline__ T pe_ld(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

struct PeView {
  int64_t nel, nface;
  int n_rows, n_up;
  const int* rows;              // sweep rows (face-point slots), upwind first
  const int32_t* elem_face;     // [4][nel]
  const double* face_jf;        // [nface]
  const double* fw;             // face Gauss weight of each face point
  const double* Gy;             // [slot][nel]
  double* Y;                    // rows of tangential points
  float* R_out;                 // mixed precision: F(uhat) - uhat at owned points (or null)
  double* partials;             // [tiles]
  IterState* it;
  double* hist;
  int max_iter;
  double tol, res_scale;
  double* uhat;                 // [2][Nqf][nface]
  __host__ __device__ const double* uhat_slot(int s, int64_t tlen) const { return uhat + s * tlen; }
};

// Hsh: the sweep rows of the operator in row order, [n_rows][NQ]. Returns true
// in the block that did the final reduction.
template <int NQ, bool CG = false>
__device__ __forceinline__ bool pe_tile(const PeView& v, const double* Hsh, const double* src,
                                        double* dst, int64_t tile, int64_t ntiles, int graph_mode,
                                        cudaGraphConditionalHandle handle) {
  constexpr int NQF = NQ / 4;
  __shared__ double red[kPeTile / 32];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t ne = v.nel, nface = v.nface;
  const int64_t e = tile * kPeTile + tid;
  double res = 0.0;
  if (e < ne) {
    double u[NQ];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int64_t face = v.elem_face[f * ne + e];
#pragma unroll
      for (int g = 0; g < NQF; ++g) u[f * NQF + g] = pe_ld<CG>(src + g * nface + face);
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      if (j >= v.n_rows) break;
      const double* Hr = Hsh + j * NQ;
      double a0 = v.Gy[j * ne + e], a1 = 0.0;
#pragma unroll
      for (int c = 0; c < NQ; c += 2) {
        a0 = fma(Hr[c], u[c], a0);
        a1 = fma(Hr[c + 1], u[c + 1], a1);
      }
      const double acc = a0 + a1;
      const int r = v.rows[j];
      if (j < v.n_up) {
        const int f = r / NQF, g = r - f * NQF;
        const int64_t face = v.elem_face[f * ne + e];
        const int64_t pt = g * nface + face;
        dst[pt] = acc;
        const double d = acc - pe_ld<CG>(src + pt);
        res += v.face_jf[face] * v.fw[g] * d * d;
        if (v.R_out) v.R_out[pt] = (float)d;
      } else {
        v.Y[(int64_t)r * ne + e] = acc;
      }
    }
  }
  // the tile's partial sum, then a ticket
  res = fsum_warp(res);
  if (lane == 0) red[wid] = res;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kPeTile / 32; ++w) s += red[w];
    v.partials[tile] = s;
    __threadfence();
    last = atomicAdd(&v.it->counter, 1u) == (unsigned int)(ntiles - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  if (wid == 0) {
    double s = 0.0;
    for (int64_t t = lane; t < ntiles; t += 32) s += reinterpret_cast<volatile double*>(v.partials)[t];
    s = fsum_warp(s);
    if (lane == 0) {
      IterState* it = v.it;
      const double r = v.res_scale * sqrt(s);
      const int k = it->k;
      if (k < v.max_iter) v.hist[k] = r;
      it->k = k + 1;
      it->r_last = r;
      it->counter = 0u;
      int cont = 1, status = EHDG_OK;
      if (!isfinite(r)) { cont = 0; status = EHDG_ERR_DIVERGED; }
      else if (r < v.tol) { cont = 0; status = EHDG_OK; }
      else if (k + 1 >= v.max_iter) { cont = 0; status = EHDG_ERR_NOT_CONVERGED; }
      it->cont = cont;
      it->status = status;
      __threadfence();
      if (graph_mode) cudaGraphSetConditional(handle, (unsigned int)cont);
    }
  }
  __syncthreads();
  return true;
}

// One 128-element tile of the FP32 correction sweep of mixed precision
// (delta_out = R + S Hy delta_in at the owned points), same shapes, one
// thread per element: the FP32 copy of the operator rows in Hsh32
// [n_rows][NQ], one FMA chain per row.
struct LpPeView {
  int64_t nel, nface;
  int n_up;
  const int* rows;
  const int32_t* elem_face;     // [4][nel]
  const float* R;               // [Nqf][nface]
  const float* in;
  float* out;
};

template <int NQ, bool CG = false>
__device__ __forceinline__ void lp_pe_tile(const LpPeView& v, const float* Hsh32, int64_t tile) {
  constexpr int NQF = NQ / 4;
  const int64_t ne = v.nel, nface = v.nface;
  const int64_t e = tile * kPeTile + threadIdx.x;
  if (e >= ne) return;
  float d[NQ];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t face = v.elem_face[f * ne + e];
#pragma unroll
    for (int g = 0; g < NQF; ++g) d[f * NQF + g] = pe_ld<CG>(v.in + g * nface + face);
  }
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    if (j >= v.n_up) break;
    const float* Hr = Hsh32 + j * NQ;
    float a = 0.f;
#pragma unroll
    for (int c = 0; c < NQ; ++c) a = fmaf(Hr[c], d[c], a);
    const int r = v.rows[j];
    const int f = r / NQF, g = r - f * NQF;
    const int64_t pt = g * nface + v.elem_face[f * ne + e];
    v.out[pt] = pe_ld<CG>(v.R + pt) + a;
  }
}

}  // namespace ehdg
