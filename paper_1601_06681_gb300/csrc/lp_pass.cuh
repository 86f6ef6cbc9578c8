// The per-warp correction pass of the mixed form for per-element transport
// operators (delta = R + S Hy delta, FP32 arithmetic on an FP32 or BF16 copy
// of the tile-major operator), built on the ring helpers of sweep_pass.cuh.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "sweep_pass.cuh"
#include "tiled_common.cuh"

namespace ehdg {

namespace {

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
