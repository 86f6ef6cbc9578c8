// Companions of the tiled transport sweep for per-element operators: the
// tile-major operator copies (built once per context), the FP32 correction
// sweep of the mixed form and the reconstruction u = G + H uhat, both
// streaming their operator rows like the sweep does (cp.async.bulk into
// per-warp mbarrier rings with bounded waits).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ehdg_internal.h"
#include "tiled_common.cuh"
#include "lp_pass.cuh"
#include "sweep_pass.cuh"

namespace ehdg {

// device allocation recorded in the context (freed by ehdg_destroy)
cudaError_t dalloc_raw(Ctx& c, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) return e;
  c.allocs.push_back(*p);
  c.bytes += (int64_t)bytes;
  return cudaSuccess;
}

namespace {

// One correction sweep per launch (mixed form, per-element operators).
template <int F, int NQF, class T>
__global__ void __launch_bounds__(32 * kTW) k_sweep_lp_tiled(const LpTParams p) {
  constexpr int NQ = F * NQF;
  constexpr int S = lp_stages<T>();
  extern __shared__ __align__(256) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar[kTW][kLSMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* stages = reinterpret_cast<T*>(tsm) + (size_t)w * S * NQ * 32;
  const uint32_t mbar0 = saddr(&mbar[w][0]);
  const int64_t nwarps = (int64_t)gridDim.x * kTW, gw = (int64_t)blockIdx.x * kTW + w;
  const int64_t J0 = p.total_rows * gw / nwarps, J1 = p.total_rows * (gw + 1) / nwarps;
  int64_t qp = 0, q_done = 0;
  ring_init(mbar0, S, lane);
  ring_fill(static_cast<const T*>(p.Hyt_lp), stages, mbar0, S, NQ, lane, J0, J1 - J0, 0, qp,
            J1 - J0);
  lp_pass<F, NQF, T, false>(p, stages, mbar0, lane, gw, J0, J1, 0, q_done, qp, J1 - J0, p.in,
                            p.out);
  ring_drain(mbar0, S, lane, q_done, qp);
}

// Reconstruction after the last iteration, u = G + H uhat (Algorithm 1
// returns the local solution for the final trace; Crank-Nicolson then takes
// u^{n+1} = 2 v - u^n), with H kept tile-major like Hy: for each tile of 32
// elements its n rows, NQFS columns x 32 elements each. Warps take equal
// contiguous ranges of the tiles' rows and stream them as the sweep does.
struct FinalTParams {
  int64_t nel, nface, ntiles, total_rows;
  int n, cn;
  const int32_t* elem_face;     // [F][nel]
  const double* Ht;             // [tile][n][NQFS][32]
  const double* uhat;           // [2][Nqf][nface]
  const IterState* it;
  const double* G;              // [n][nel]
  double* u;                    // [n][nel]
  int* err;
};

template <int F, int NQF>
__global__ void __launch_bounds__(32 * kTW, (F * NQF <= 28) ? EHDG_TILED_MINB : 1)
    k_final_tiled(const FinalTParams p) {
  constexpr int NQ = F * NQF;
  constexpr uint32_t kRowBytes = (uint32_t)NQ * 32u * 8u;
  extern __shared__ __align__(256) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar[kTW][kTS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* stages = reinterpret_cast<double*>(tsm) + (size_t)w * kTS * NQ * 32;
  if (lane == 0) {
    for (int s = 0; s < kTS; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[w][s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();

  const int64_t ne = p.nel, nface = p.nface;
  const double* src = p.uhat + (int64_t)((p.it->k + 1) & 1) * NQF * nface;
  const int64_t nwarps = (int64_t)gridDim.x * kTW, gw = (int64_t)blockIdx.x * kTW + w;
  const int64_t J0 = p.total_rows * gw / nwarps, J1 = p.total_rows * (gw + 1) / nwarps;
  int64_t Jp = J0;
  for (int s = 0; s < kTS && Jp < J1; ++s, ++Jp)
    if (lane == 0)
      issue_row(saddr(&mbar[w][s]), saddr(stages + (size_t)s * NQ * 32), p.Ht + Jp * NQ * 32,
                kRowBytes);

  int64_t t = J0 / p.n;
  int r = (int)(J0 - t * p.n);
  int fid_n[F];
  auto load_faces = [&](int64_t tt) {
    const int64_t ee = tt * 32 + lane;
#pragma unroll
    for (int f = 0; f < F; ++f)
      fid_n[f] = (tt < p.ntiles && ee < ne) ? p.elem_face[(int64_t)f * ne + ee] : 0;
  };
  if (J0 < J1) load_faces(t);
  double u[NQ];
  int64_t e = 0;
  bool fresh = true;
  int64_t J = J0;
  for (; J < J1; ++J) {
    if (fresh) {
      e = t * 32 + lane;
#pragma unroll
      for (int f = 0; f < F; ++f)
#pragma unroll
        for (int g = 0; g < NQF; ++g)
          u[f * NQF + g] = e < ne ? src[(int64_t)g * nface + fid_n[f]] : 0.0;
      fresh = false;
    }
    const bool live = e < ne;
    const int64_t at = (int64_t)r * ne + e;
    const double g0 = live ? p.G[at] : 0.0;           // used after the FMA chain
    const double uold = (live && p.cn) ? p.u[at] : 0.0;
    if (++r == p.n) {
      r = 0;
      ++t;
      fresh = true;
      if (J + 1 < J1) load_faces(t);
    }
    const int st = (int)((J - J0) % kTS);
    if (!wait_phase_warp(saddr(&mbar[w][st]), (uint32_t)(((J - J0) / kTS) & 1))) {
      if (lane == 0) atomicExch(p.err, 1);
      break;
    }
    const double* Hs = stages + (size_t)st * NQ * 32;
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < NQ; ++c) acc = fma(Hs[c * 32 + lane], u[c], acc);
    __syncwarp();                                // every lane has read the stage
    if (Jp < J1) {
      if (lane == 0)
        issue_row(saddr(&mbar[w][st]), saddr(stages + (size_t)st * NQ * 32),
                  p.Ht + Jp * NQ * 32, kRowBytes);
      ++Jp;
    }
    acc += g0;
    if (live) p.u[at] = p.cn ? 2.0 * acc - uold : acc;
  }
  for (int64_t Jw = J; Jw < Jp; ++Jw) {
    const int st = (int)((Jw - J0) % kTS);
    if (lane == 0) wait_phase(saddr(&mbar[w][st]), (uint32_t)(((Jw - J0) / kTS) & 1));
  }
  __syncwarp();
}

// Trace index g * nface + face of the point each (slot, element) row
// produces; slots past an element's rows hold 0.
__global__ void k_row_points(int64_t nel, int NQFS, int Nqf, int64_t nface,
                             const uint8_t* rowid, const uint8_t* nrows,
                             const int32_t* elem_face, int32_t* ptid) {
  const int64_t total = (int64_t)NQFS * nel;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / nel);
    const int64_t e = i - (int64_t)j * nel;
    int32_t v = 0;
    if (j < nrows[e]) {
      const int r = rowid[i];
      const int f = r / Nqf, g = r - f * Nqf;
      v = (int32_t)((int64_t)g * nface + elem_face[(int64_t)f * nel + e]);
    }
    ptid[i] = v;
  }
}

// Low-precision copy of the tile-major rows (nq x 32 values each) in the
// correction sweep's pair-interleaved order: FP32, or BF16 rounded to
// nearest even through FP32.
__device__ __forceinline__ void put_lp(float* d, double v) { *d = (float)v; }
__device__ __forceinline__ void put_lp(__nv_bfloat16* d, double v) {
  *d = __float2bfloat16_rn((float)v);
}

template <class T>
__global__ void k_round_rows(int64_t n, int nq, const double* src, T* dst) {
  const int64_t row_len = (int64_t)nq * 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / row_len, w = i - r * row_len;
    const int c = (int)(w >> 5), lane = (int)(w & 31);
    put_lp(dst + r * row_len + pair_index(c, lane), src[i]);
  }
}

// Tile-major copy of the reconstruction operator H ([n][NQFS][nel] ->
// [tile][n][NQFS][32], zero past the last element).
__global__ void k_tile_h(int64_t nel, int n, int nq, int64_t ntiles, const double* H, double* Ht) {
  const int64_t total = ntiles * n * nq * 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i & 31);
    const int64_t rest = i >> 5;                 // (tile * n + r) * nq + c
    const int c = (int)(rest % nq);
    const int64_t tr = rest / nq;
    const int r = (int)(tr % n);
    const int64_t tile = tr / n;
    const int64_t e = tile * 32 + l;
    Ht[i] = e < nel ? H[((int64_t)r * nq + c) * nel + e] : 0.0;
  }
}

// Tile-major copy of the compacted per-element rows; rows an element does not
// use are zero, as are the lanes past the last element.
__global__ void k_tile_hy(int64_t nel, int nq, int64_t ntiles, const int32_t* tile_row0,
                          const uint8_t* tile_nrows, const uint8_t* nrows, const double* Hy,
                          double* Hyt) {
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int n = tile_nrows[t] * nq * 32;
    double* out = Hyt + (int64_t)tile_row0[t] * nq * 32;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int l = i & 31, jc = i >> 5;
      const int j = jc / nq, c = jc - j * nq;
      const int64_t e = t * 32 + l;
      out[i] = (e < nel && j < nrows[e]) ? Hy[((int64_t)j * nq + c) * nel + e] : 0.0;
    }
  }
}

template <int F, int NQF>
cudaError_t final_config(int64_t total_rows, int64_t ntiles, int* grid, size_t* smem_out) {
  return tiled_shape_of(k_final_tiled<F, NQF>, F * NQF, total_rows, ntiles, grid, smem_out);
}

template <int F, int NQF>
cudaError_t final_launch(const FinalTParams& p, int grid, size_t smem, cudaStream_t s) {
  k_final_tiled<F, NQF><<<grid, 32 * kTW, smem, s>>>(p);
  return cudaGetLastError();
}

// the FP32 sweep runs on the FP64 sweep's grid (same warps, same row ranges)
template <int F, int NQF, class T>
cudaError_t lp_config(int64_t total_rows, int64_t ntiles, int* grid, size_t* smem_out) {
  return tiled_shape_of(k_sweep_lp_tiled<F, NQF, T>, F * NQF, total_rows, ntiles, grid, smem_out,
                        sizeof(T) * lp_stages<T>());
}

template <int F, int NQF, class T>
cudaError_t lp_launch(const LpTParams& p, int grid, size_t smem, cudaStream_t s) {
  k_sweep_lp_tiled<F, NQF, T><<<grid, 32 * kTW, smem, s>>>(p);
  return cudaGetLastError();
}

struct AuxOps {
  cudaError_t (*final_config)(int64_t, int64_t, int*, size_t*);
  cudaError_t (*final_launch)(const FinalTParams&, int, size_t, cudaStream_t);
  cudaError_t (*lp_config)(int64_t, int64_t, int*, size_t*);
  cudaError_t (*lp_launch)(const LpTParams&, int, size_t, cudaStream_t);
  cudaError_t (*lp16_config)(int64_t, int64_t, int*, size_t*);
  cudaError_t (*lp16_launch)(const LpTParams&, int, size_t, cudaStream_t);
};

bool aux_ops(int F, int Nqf, AuxOps* out) {
#define EHDG_AUX_CASE(f_, q_)                                                             \
  if (F == f_ && Nqf == q_) {                                                             \
    *out = AuxOps{&final_config<f_, q_>, &final_launch<f_, q_>, &lp_config<f_, q_, float>,  \
                  &lp_launch<f_, q_, float>, &lp_config<f_, q_, __nv_bfloat16>,            \
                  &lp_launch<f_, q_, __nv_bfloat16>};                                     \
    return true;                                                                          \
  }
  EHDG_TILED_SHAPES(EHDG_AUX_CASE)
#undef EHDG_AUX_CASE
  return false;
}

}  // namespace

cudaError_t build_tiled_operator(Ctx& c) {
  const int64_t ntiles = (c.nel + 31) / 32;
  std::vector<uint8_t> nr((size_t)c.nel);
  cudaError_t err = cudaMemcpy(nr.data(), c.nrows, (size_t)c.nel, cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return err;
  std::vector<uint8_t> tnr((size_t)ntiles, 0);
  std::vector<int32_t> row0((size_t)ntiles, 0);
  int64_t rows = 0;
  for (int64_t t = 0; t < ntiles; ++t) {
    uint8_t m = 0;
    for (int64_t e = t * 32; e < std::min<int64_t>(c.nel, t * 32 + 32); ++e) m = std::max(m, nr[e]);
    tnr[t] = m;
    row0[t] = (int32_t)rows;
    rows += m;
  }
  if (rows > INT32_MAX) return cudaErrorInvalidValue;
  c.ntiles = ntiles;
  c.tile_rows = rows;
  if ((err = dalloc_raw(c, (void**)&c.tile_nrows, (size_t)ntiles)) != cudaSuccess) return err;
  if ((err = dalloc_raw(c, (void**)&c.tile_row0, sizeof(int32_t) * (size_t)ntiles)) != cudaSuccess)
    return err;
  if ((err = dalloc_raw(c, (void**)&c.Hyt, sizeof(double) * (size_t)std::max<int64_t>(rows, 1) *
                                                c.NQFS * 32)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpy(c.tile_nrows, tnr.data(), (size_t)ntiles, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return err;
  if ((err = cudaMemcpy(c.tile_row0, row0.data(), sizeof(int32_t) * (size_t)ntiles,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  // launch shape, fixed for the context, and the tile of each warp's first row
  AuxOps ops;
  if (!aux_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  if ((err = tiled_sweep_shape(c, rows, ntiles, &c.tiled_grid, &c.tiled_smem)) != cudaSuccess)
    return err;
  const int64_t nwarps = (int64_t)c.tiled_grid * kTW;
  std::vector<int32_t> wt((size_t)nwarps, 0);
  for (int64_t gw = 0, tt = 0; gw < nwarps; ++gw) {
    const int64_t J0 = rows * gw / nwarps;
    while (tt + 1 < ntiles && row0[tt + 1] <= J0) ++tt;   // last tile starting at or before J0
    wt[gw] = (int32_t)tt;
  }
  if ((err = dalloc_raw(c, (void**)&c.tiled_warp_tile, sizeof(int32_t) * (size_t)nwarps)) !=
      cudaSuccess)
    return err;
  // the persistent form runs on the same grid; it needs every block resident
  c.persist_fits = (int64_t)tiled_persist_blocks_per_sm(c) * device_sms() >= c.tiled_grid;
  if ((err = dalloc_raw(c, (void**)&c.ppartials, sizeof(double) * 2 * (size_t)c.tiled_grid)) !=
      cudaSuccess)
    return err;
  if ((err = cudaMemcpy(c.tiled_warp_tile, wt.data(), sizeof(int32_t) * (size_t)nwarps,
                        cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  int grid = (int)std::min<int64_t>(ntiles, 152 * 16);
  k_tile_hy<<<grid < 1 ? 1 : grid, 256, 0, c.stream>>>(c.nel, c.NQFS, ntiles, c.tile_row0,
                                                       c.tile_nrows, c.nrows, c.Hy, c.Hyt);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  // reconstruction operator, all n rows of every tile
  const int64_t hrows = ntiles * c.n;
  if ((err = dalloc_raw(c, (void**)&c.Ht, sizeof(double) * (size_t)hrows * c.NQFS * 32)) !=
      cudaSuccess)
    return err;
  if ((err = ops.final_config(hrows, ntiles, &c.ftiled_grid, &c.ftiled_smem)) != cudaSuccess)
    return err;
  k_tile_h<<<152 * 8, 256, 0, c.stream>>>(c.nel, c.n, c.NQFS, ntiles, c.H, c.Ht);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (c.mixed) {
    // the trace index of every row's point (the correction sweeps prefetch it)
    if ((int64_t)c.Nqf * c.nface > INT32_MAX) return cudaErrorInvalidValue;
    if ((err = dalloc_raw(c, (void**)&c.ptid, sizeof(int32_t) * (size_t)c.NQFS * c.nel)) !=
        cudaSuccess)
      return err;
    k_row_points<<<152 * 8, 256, 0, c.stream>>>(c.nel, c.NQFS, c.Nqf, c.nface, c.rowid, c.nrows,
                                                c.geo.elem_face, c.ptid);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // low-precision copy of the tile-major sweep operator for the correction
    // sweeps: BF16 for MIXED_BF16, FP32 otherwise
    const int64_t nlp = std::max<int64_t>(rows * c.NQFS * 32, 1);
    if (c.precision == EHDG_MIXED_BF16) {
      if ((err = dalloc_raw(c, (void**)&c.Hyt16, sizeof(__nv_bfloat16) * (size_t)nlp)) !=
          cudaSuccess)
        return err;
      k_round_rows<<<152 * 8, 256, 0, c.stream>>>(rows * c.NQFS * 32, c.NQFS, c.Hyt,
                                                  static_cast<__nv_bfloat16*>(c.Hyt16));
    } else {
      if ((err = dalloc_raw(c, (void**)&c.Hyt32, sizeof(float) * (size_t)nlp)) != cudaSuccess)
        return err;
      k_round_rows<<<152 * 8, 256, 0, c.stream>>>(rows * c.NQFS * 32, c.NQFS, c.Hyt, c.Hyt32);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // the correction sweep's own launch shape (its shared memory allows more
    // warps than the FP64 sweep's) and the tile of each of its warps' first row
    AuxOps ops2;
    if (!aux_ops(c.F, c.Nqf, &ops2)) return cudaErrorInvalidValue;
    if ((err = (c.Hyt16 ? ops2.lp16_config : ops2.lp_config)(rows, ntiles, &c.lp_grid,
                                                             &c.lp_smem)) != cudaSuccess)
      return err;
    const int64_t lwarps = (int64_t)c.lp_grid * kTW;
    std::vector<int32_t> lt((size_t)lwarps, 0);
    for (int64_t gw = 0, tt = 0; gw < lwarps; ++gw) {
      const int64_t J0 = rows * gw / lwarps;
      while (tt + 1 < ntiles && row0[tt + 1] <= J0) ++tt;
      lt[gw] = (int32_t)tt;
    }
    if ((err = dalloc_raw(c, (void**)&c.lp_warp_tile, sizeof(int32_t) * (size_t)lwarps)) !=
        cudaSuccess)
      return err;
    if ((err = cudaMemcpy(c.lp_warp_tile, lt.data(), sizeof(int32_t) * (size_t)lwarps,
                          cudaMemcpyHostToDevice)) != cudaSuccess)
      return err;
  }
  return cudaSuccess;
}

cudaError_t launch_lp_sweep_tiled(Ctx& c, const float* in, float* out) {
  LpTParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.ntiles = c.ntiles;
  p.total_rows = c.tile_rows;
  p.warp_tile = c.lp_warp_tile;
  p.tile_row0 = c.tile_row0;
  p.tile_nrows = c.tile_nrows;
  p.rowid = c.rowid;
  p.nrows = c.nrows;
  p.nup = c.nup;
  p.elem_face = c.geo.elem_face;
  p.ptid = c.ptid;
  p.Hyt_lp = c.Hyt16 ? c.Hyt16 : static_cast<const void*>(c.Hyt32);
  p.R = c.R32;
  p.in = in;
  p.out = out;
  p.Y32 = c.Y32;
  p.err = c.tc_err;
  AuxOps ops;
  if (!aux_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  return c.Hyt16 ? ops.lp16_launch(p, c.lp_grid, c.lp_smem, c.stream)
                 : ops.lp_launch(p, c.lp_grid, c.lp_smem, c.stream);
}

cudaError_t launch_final_tiled(Ctx& c) {
  FinalTParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.ntiles = c.ntiles;
  p.total_rows = c.ntiles * c.n;
  p.n = c.n;
  p.cn = (c.scheme == EHDG_CN) ? 1 : 0;
  p.elem_face = c.geo.elem_face;
  p.Ht = c.Ht;
  p.uhat = c.uhat;
  p.it = c.it;
  p.G = c.G;
  p.u = c.u;
  p.err = c.tc_err;
  AuxOps ops;
  if (!aux_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  return ops.final_launch(p, c.ftiled_grid, c.ftiled_smem, c.stream);
}

}  // namespace ehdg
