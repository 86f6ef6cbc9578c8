// One 32-element tile of the fused FP64 transport sweep with a local operator
// shared by every element (Sec. 3, eqs. transportLocalk1 and
// transportLocale): gather the tile's traces at its elements' face points,
// form every sweep row Y = Gy + Hy uhat as one thread's FMA chain (even and
// odd columns in two chains), and let the upwind element write the new trace
// at the points it owns, adding w (uhat^{k+1} - uhat^k)^2 to its residual
// share. The single-problem sweep and the batched loop both run this code,
// so an instance's iterates do not depend on which of them ran it.
#pragma once

#include <cuda_runtime.h>

#include "ehdg_internal.h"

namespace ehdg {

struct FusedTileView {
  int64_t nel, nface;
  int NQFS, Nqf, F, n_rows, n_up;
  const int* rows;              // sweep rows (face-point slots), upwind first
  const int32_t* elem_face;     // [F][nel]
  const double* face_jf;        // [nface]
  const double* fw;             // face Gauss weight of each face point
  const double* Gy;             // [slot][nel]
  double* Y;                    // rows of tangential points
  float* R_out;                 // mixed precision: F(uhat) - uhat at owned points (or null)
};

// Threads: lane = threadIdx.x (element of the tile), t = threadIdx.y (row
// group, FT of them). Hsh: the operator rows [NQFS][NQFS]; uh [NQFS][32] and
// fid [F][32]: shared scratch of the block.
template <int NQ, int FT>
__device__ __forceinline__ void fused_tile_shared(const FusedTileView& v, const double* Hsh,
                                                  double* uh, int* fid, const double* src,
                                                  double* dst, int64_t tile, double& acc_res) {
  const int nq = NQ > 0 ? NQ : v.NQFS;
  const int lane = threadIdx.x, t = threadIdx.y;
  const int64_t ne = v.nel, nface = v.nface;
  const int64_t e = tile * 32 + lane;
  __syncthreads();                                      // previous tile done with uh/fid
  if (e < ne) {
    for (int f = t; f < v.F; f += FT) fid[f * 32 + lane] = v.elem_face[f * ne + e];
  }
  __syncthreads();
  if (e < ne) {
    for (int i = t; i < nq; i += FT) {
      const int f = i / v.Nqf, g = i - f * v.Nqf;
      uh[i * 32 + lane] = src[g * nface + fid[f * 32 + lane]];
    }
  }
  __syncthreads();
  if (e < ne) {
    for (int j = t; j < v.n_rows; j += FT) {
      // two independent FMA chains (even and odd columns)
      double a0 = v.Gy[j * ne + e], a1 = 0.0;
      const int r = v.rows[j];
      const double* Hr = Hsh + r * nq;
      if constexpr (NQ > 0) {
#pragma unroll 16
        for (int c = 0; c < NQ; c += 2) {
          a0 = fma(Hr[c], uh[c * 32 + lane], a0);
          if (c + 1 < NQ) a1 = fma(Hr[c + 1], uh[(c + 1) * 32 + lane], a1);
        }
      } else {
        for (int c = 0; c < nq; ++c) a0 = fma(Hr[c], uh[c * 32 + lane], a0);
      }
      const double acc = a0 + a1;
      if (j < v.n_up) {
        const int f = r / v.Nqf, g = r - f * v.Nqf;
        const int face = fid[f * 32 + lane];
        dst[g * nface + face] = acc;
        const double d = acc - uh[r * 32 + lane];
        acc_res += v.face_jf[face] * v.fw[g] * d * d;
        if (v.R_out) v.R_out[g * nface + face] = (float)d;
      } else {
        v.Y[(int64_t)r * ne + e] = acc;
      }
    }
  }
}

}  // namespace ehdg
