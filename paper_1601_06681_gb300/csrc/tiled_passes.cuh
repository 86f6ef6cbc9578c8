// The per-warp row passes of the tiled per-element transport kernels: the
// FP64 sweep pass (local solve folded into Hy, upwind trace formula with
// owner writes, residual share; Sec. 3, eqs. transportLocalk1 and
// transportLocale) and the low-precision correction pass of the mixed form.
// Each warp streams its rows through a ring of shared-memory stages filled by
// cp.async.bulk, one mbarrier per stage, every wait bounded.
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

// Low-precision correction sweep of the mixed form (delta = R + S Hy delta,
// the correction equation of the FP64 trace fixed point), FP32 arithmetic on
// the CUDA cores with an FP32 or BF16 copy of the tile-major operator. Same
// row ranges and warp starts as the FP64 sweep; rows are 2x (FP32) or 4x
// (BF16) shorter, so each warp keeps that many more stages in the same
// shared memory. Owned points: out = R + row value;
// rows of points with beta.n = 0 go to Y32 for the finishing kernel.
// stages per warp of the correction sweep (rows of FP32 or BF16)
template <class T>
__host__ __device__ constexpr int lp_stages() {
  return 4;
}
constexpr int kLSMax = 4;

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// two adjacent values of a pair-interleaved row as FP32
__device__ __forceinline__ float2 load_pair(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}
__device__ __forceinline__ float2 load_pair(const __nv_bfloat16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}

// index of (column c, lane) in a pair-interleaved row of nq x 32 values
__host__ __device__ __forceinline__ int64_t pair_index(int c, int lane) {
  return ((int64_t)(c >> 1) * 32 + lane) * 2 + (c & 1);
}

struct LpTParams {
  int64_t nel, nface, ntiles, total_rows;
  const int32_t* warp_tile;
  const int32_t* tile_row0;
  const uint8_t* tile_nrows;
  const uint8_t* rowid;
  const uint8_t* nrows;
  const uint8_t* nup;
  const int32_t* elem_face;
  const int32_t* ptid;          // [slot][nel] trace index g * nface + face of each row's point
  const void* Hyt_lp;           // tile-major rows, FP32 or BF16
  const float* R;               // [Nqf][nface]
  const float* in;
  float* out;
  float* Y32;                   // [NQFS][nel]
  int* err;
};

// Position of a warp in its row sequence: tile t, slot j, rows of the tile.
struct RowPos {
  int64_t t;
  int j, nr;
};

template <class P>
__device__ __forceinline__ void rowpos_next(const P& p, RowPos& r) {
  if (++r.j == r.nr) {
    r.j = 0;
    do {
      ++r.t;
    } while (r.t < p.ntiles && p.tile_nrows[r.t] == 0);
    r.nr = r.t < p.ntiles ? p.tile_nrows[r.t] : 0;
  }
}

// One correction pass of a warp over its rows (FP32 arithmetic): owned
// points get out = R + row value, rows of points with beta.n = 0 go to Y32.
// The correction has a short FMA chain, so the pass is bound by the latency
// of its dependent loads. Each row's trace index is loaded two rows ahead and
// its R value one row ahead. CG: the input trace is read through L2 only
// (persistent launches).
template <int F, int NQF, class T, bool CG>
__device__ __forceinline__ bool lp_pass(const LpTParams& p, T* stages, uint32_t mbar0, int lane,
                                        int64_t gw, int64_t J0, int64_t J1, int64_t q0,
                                        int64_t& q_done, int64_t& qp, int64_t qp_end,
                                        const float* in, float* out) {
  constexpr int NQ = F * NQF;
  constexpr int S = lp_stages<T>();
  const T* rows = static_cast<const T*>(p.Hyt_lp);
  const int64_t ne = p.nel, nface = p.nface;
  const int64_t L = J1 - J0;
  if (L <= 0) return true;
  auto ptid_at = [&](const RowPos& r) -> int {
    const int64_t ee = r.t * 32 + lane;
    return (r.t < p.ntiles && ee < ne) ? p.ptid[(int64_t)r.j * ne + ee] : 0;
  };
  RowPos cur;
  cur.t = p.warp_tile[gw];
  cur.j = (int)(J0 - p.tile_row0[cur.t]);
  cur.nr = p.tile_nrows[cur.t];
  RowPos ahead1 = cur, ahead2 = cur;
  rowpos_next(p, ahead1);
  ahead2 = ahead1;
  rowpos_next(p, ahead2);
  int pt_cur = ptid_at(cur);
  int pt_nxt = L > 1 ? ptid_at(ahead1) : 0;
  float rv_cur = CG ? __ldcg(p.R + pt_cur) : p.R[pt_cur];
  int nr_e = 0, nu_e = 0;
  int64_t e = 0, t_gathered = -1;
  float d[NQ];
  // face ids of the tile the next row enters, loaded a row early
  int fid_n[F];
  int64_t fid_tile = -1;
  int rid_n = (cur.t * 32 + lane < ne) ? p.rowid[(int64_t)cur.j * ne + cur.t * 32 + lane] : 0;
  for (int64_t i = 0; i < L; ++i) {
    if (cur.t != t_gathered) {
      // the tile's correction values at each element's face points
      e = cur.t * 32 + lane;
      const bool live = e < ne;
      nr_e = live ? p.nrows[e] : 0;
      nu_e = live ? p.nup[e] : 0;
      const bool have = fid_tile == cur.t;
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const int fid = have ? fid_n[f] : (live ? p.elem_face[(int64_t)f * ne + e] : 0);
#pragma unroll
        for (int g = 0; g < NQF; ++g) {
          const float* a = in + (int64_t)g * nface + fid;
          d[f * NQF + g] = live ? (CG ? __ldcg(a) : *a) : 0.f;
        }
      }
      t_gathered = cur.t;
    }
    const int j = cur.j;
    const bool row_live = j < nr_e;
    const bool owned = row_live && j < nu_e;
    const int pt = pt_cur;
    const float rv = rv_cur;
    const int rid = rid_n;
    // prefetch: R of the next row, the trace index of the row after it
    float rv_nxt = 0.f;
    if (i + 1 < L) rv_nxt = CG ? __ldcg(p.R + pt_nxt) : p.R[pt_nxt];
    int pt_nn = 0;
    if (i + 2 < L) pt_nn = ptid_at(ahead2);
    // the next row's position and point id
    cur = ahead1;
    ahead1 = ahead2;
    if (i + 2 < L) rowpos_next(p, ahead2);
    if (i + 1 < L && cur.t * 32 + lane < ne) rid_n = p.rowid[(int64_t)cur.j * ne + cur.t * 32 + lane];
    if (i + 1 < L && cur.t != t_gathered && fid_tile != cur.t) {
      const int64_t ee = cur.t * 32 + lane;
#pragma unroll
      for (int f = 0; f < F; ++f)
        fid_n[f] = (cur.t < p.ntiles && ee < ne) ? p.elem_face[(int64_t)f * ne + ee] : 0;
      fid_tile = cur.t;
    }

    const int64_t q = q0 + i;
    const int st = (int)(q % S);
    if (!wait_phase_warp(mbar0 + 8u * st, (uint32_t)((q / S) & 1))) {
      if (lane == 0) atomicExch(p.err, 1);
      return false;
    }
    q_done = q + 1;
    // the copy is pair-interleaved: columns 2h and 2h+1 of a lane are adjacent
    const T* Hs = stages + (size_t)st * NQ * 32;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int c = 0; c < NQ; c += 2) {
      const float2 h = load_pair(Hs + ((c >> 1) * 32 + lane) * 2);
      a0 = fmaf(h.x, d[c], a0);
      a1 = fmaf(h.y, d[c + 1], a1);
    }
    const float acc = a0 + a1;
    __syncwarp();                                // every lane has read the stage
    ring_fill(rows, stages, mbar0, S, NQ, lane, J0, L, q_done, qp, qp_end);
    if (owned) {
      out[pt] = rv + acc;
    } else if (row_live) {
      p.Y32[(int64_t)rid * ne + e] = acc;
    }
    pt_cur = pt_nxt;
    rv_cur = rv_nxt;
    pt_nxt = pt_nn;
  }
  return true;
}

}  // namespace

}  // namespace ehdg
