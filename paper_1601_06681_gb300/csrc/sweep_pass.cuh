// The per-warp FP64 row pass of the tiled per-element transport kernels
// (local solve folded into Hy, upwind trace formula with owner writes,
// residual share; Sec. 3, eqs. transportLocalk1 and transportLocale), and the
// ring helpers that every tiled kernel uses: each warp streams its rows
// through a ring of shared-memory stages filled by cp.async.bulk, one
// mbarrier per stage, every wait bounded.
//
// Ring bookkeeping: sequence number q holds row J0 + (q mod L), L = J1 - J0,
// in stage q mod S and completes phase (q / S) & 1 of that stage's mbarrier.
// q_done counts the sequence numbers consumed, qp the ones issued; a pass
// consumes L consecutive sequence numbers, and the producer runs up to S
// ahead of the consumer but never past qp_end.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "tiled_common.cuh"

namespace ehdg {

namespace {

__device__ __forceinline__ void ring_init(uint32_t mbar0, int S, int lane) {
  if (lane == 0) {
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8u * s));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
}

// issue copies while the ring has a free stage and qp < qp_end
template <class T>
__device__ __forceinline__ void ring_fill(const T* rows, T* stages, uint32_t mbar0, int S, int NQ,
                                          int lane, int64_t J0, int64_t L, int64_t q_done,
                                          int64_t& qp, int64_t qp_end) {
  const uint32_t bytes = (uint32_t)NQ * 32u * (uint32_t)sizeof(T);
  while (qp < q_done + S && qp < qp_end) {
    const int s = (int)(qp % S);
    if (lane == 0)
      issue_row(mbar0 + 8u * s, saddr(stages + (size_t)s * NQ * 32), rows + (J0 + qp % L) * NQ * 32,
                bytes);
    ++qp;
  }
}

// copies still in flight (a speculative prefetch that will not be consumed,
// or after a wait gave up): wait for them, bounded
__device__ __forceinline__ void ring_drain(uint32_t mbar0, int S, int lane, int64_t q_done,
                                           int64_t qp) {
  for (int64_t q = q_done; q < qp; ++q)
    if (lane == 0) wait_phase(mbar0 + 8u * (uint32_t)(q % S), (uint32_t)((q / S) & 1));
  __syncwarp();
}

struct TiledParams {
  int64_t nel, nface, ntiles, total_rows;
  const int32_t* warp_tile;      // [grid * kTW] tile holding each warp's first row
  const uint8_t* rowid;          // [slot][nel]
  const uint8_t* nrows;          // [nel]
  const uint8_t* nup;            // [nel]
  const int32_t* elem_face;      // [F][nel]
  const double* face_jf;
  double fw[kMaxQ * kMaxQ];
  const double* Hyt;             // tile-major rows
  const int32_t* tile_row0;      // [ntiles] first row of each tile in Hyt
  const uint8_t* tile_nrows;     // [ntiles] rows of each tile
  double* uhat;                  // [2][Nqf][nface]
  IterState* it;
  const double* Gy;              // [slot][nel]
  double* Y;                     // [NQFS][nel]
  float* R_out;
  double* partials;
  int final_here;
  double tol, res_scale;
  int max_iter;
  double* hist;
  int graph_mode;
  cudaGraphConditionalHandle handle;
  int* err;
};

// One pass of a warp over its rows J0 .. J1-1 (so every warp has the same
// work to within one row, whatever the tile boundaries). The rows go through
// the warp's ring of kTS stages: ring sequence number q holds row
// J0 + (q mod L), L = J1 - J0, in stage q mod kTS, and completes mbarrier phase
// (q / kTS) & 1 of that stage. This pass consumes q0 .. q0 + L - 1; the
// producer cursor qp (kTS ahead of the consumer) issues up to qp_end, so a
// persistent caller keeps streaming the next pass's rows. CG: the trace is
// read through L2 only (it is rewritten by other SMs during a persistent
// launch). Returns false if a bounded wait gave up.
template <int F, int NQF, bool CG>
__device__ __forceinline__ bool sweep_pass(const TiledParams& p, double* stages, uint32_t mbar0,
                                           int lane, int64_t gw, int64_t J0, int64_t J1,
                                           int64_t q0, int64_t& q_done, int64_t& qp,
                                           int64_t qp_end, const double* src, double* dst,
                                           double& acc_res) {
  constexpr int NQ = F * NQF;
  const int64_t ne = p.nel, nface = p.nface;
  const int64_t L = J1 - J0;
  if (L <= 0) return true;
  int64_t t = p.warp_tile[gw];
  int j = (int)(J0 - p.tile_row0[t]);
  int nr_t = 0, nr_e = 0, nu_e = 0;
  int64_t e = 0;
  int fid[F];
  double jf[F], u[NQ];
  // per-tile values of tile t, loaded as soon as t is known (one row before
  // the warp enters the tile): face ids, row counts
  int fid_n[F], nr_e_n = 0, nu_e_n = 0, nr_t_n = 0;
  auto load_tile = [&](int64_t tt) {
    const int64_t ee = tt * 32 + lane;
    const bool live = tt < p.ntiles && ee < ne;
    nr_t_n = tt < p.ntiles ? p.tile_nrows[tt] : 0;
#pragma unroll
    for (int f = 0; f < F; ++f) fid_n[f] = live ? p.elem_face[(int64_t)f * ne + ee] : 0;
    nr_e_n = live ? p.nrows[ee] : 0;
    nu_e_n = live ? p.nup[ee] : 0;
  };
  load_tile(t);
  bool fresh = true;                             // tile t not gathered yet
  // the next row's Gy value and point id are loaded one row ahead (slots
  // beyond an element's rows exist in both arrays and are never used)
  double gy_n = 0.0;
  int rid_n = 0;
  if (t * 32 + lane < ne) {
    gy_n = p.Gy[(int64_t)j * ne + t * 32 + lane];
    rid_n = p.rowid[(int64_t)j * ne + t * 32 + lane];
  }
  for (int64_t i = 0; i < L; ++i) {
    if (fresh) {
      // the element's faces, their Jacobians and uhat^k at its face points
      e = t * 32 + lane;
      const bool live = e < ne;
      nr_t = nr_t_n;
      nr_e = nr_e_n;
      nu_e = nu_e_n;
#pragma unroll
      for (int f = 0; f < F; ++f) fid[f] = fid_n[f];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        jf[f] = live ? p.face_jf[fid[f]] : 0.0;
#pragma unroll
        for (int g = 0; g < NQF; ++g) {
          const double* a = src + (int64_t)g * nface + fid[f];
          u[f * NQF + g] = live ? (CG ? __ldcg(a) : *a) : 0.0;
        }
      }
      fresh = false;
    }
    const bool row_live = j < nr_e;
    const double gy = gy_n;
    const int rid = rid_n;
    const int j_cur = j;
    // advance to the next row (and tile) and start its Gy / point-id loads
    if (++j == nr_t) {
      j = 0;
      do {
        ++t;
      } while (t < p.ntiles && p.tile_nrows[t] == 0);
      fresh = true;
      if (i + 1 < L) load_tile(t);
    }
    if (i + 1 < L && t * 32 + lane < ne) {
      gy_n = p.Gy[(int64_t)j * ne + t * 32 + lane];
      rid_n = p.rowid[(int64_t)j * ne + t * 32 + lane];
    }

    const int64_t q = q0 + i;
    const int st = (int)(q % kTS);
    if (!wait_phase_warp(mbar0 + 8u * st, (uint32_t)((q / kTS) & 1))) {
      if (lane == 0) atomicExch(p.err, 1);
      return false;
    }
    q_done = q + 1;
    const double* Hs = stages + (size_t)st * NQ * 32;
    double a[kCH];
    a[0] = row_live ? gy : 0.0;
#pragma unroll
    for (int c2 = 1; c2 < kCH; ++c2) a[c2] = 0.0;
#pragma unroll
    for (int c = 0; c < NQ; ++c) a[c % kCH] = fma(Hs[c * 32 + lane], u[c], a[c % kCH]);
    double acc = a[0];
    if constexpr (kCH == 2) acc = a[0] + a[1];
    if constexpr (kCH == 4) acc = (a[0] + a[1]) + (a[2] + a[3]);
    __syncwarp();                                // every lane has read the stage
    ring_fill(p.Hyt, stages, mbar0, kTS, NQ, lane, J0, L, q_done, qp, qp_end);
    if (row_live) {
      const int f = rid / NQF, g = rid - f * NQF;
      int face = 0;
      double jfv = 0.0, uk = 0.0;
#pragma unroll
      for (int q2 = 0; q2 < F; ++q2)
        if (q2 == f) {
          face = fid[q2];
          jfv = jf[q2];
        }
#pragma unroll
      for (int c = 0; c < NQ; ++c)
        if (c == rid) uk = u[c];
      if (j_cur < nu_e) {
        const int64_t pt = (int64_t)g * nface + face;
        dst[pt] = acc;
        const double d = acc - uk;
        acc_res = fma(jfv * p.fw[g] * d, d, acc_res);
        if (p.R_out) p.R_out[pt] = (float)d;
      } else {
        p.Y[(int64_t)rid * ne + e] = acc;
      }
    }
  }
  return true;
}

}  // namespace

}  // namespace ehdg
