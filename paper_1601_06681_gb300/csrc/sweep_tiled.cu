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

#include <vector>

#include "ehdg_internal.h"
#include "sweep_common.cuh"

namespace ehdg {

namespace {

// compile-time tuning: warps per block (independent of each other), stages
// per warp, independent FMA chains per row
#ifndef EHDG_TILED_TW
#define EHDG_TILED_TW 4
#endif
#ifndef EHDG_TILED_TS
#define EHDG_TILED_TS 2
#endif
#ifndef EHDG_TILED_CH
#define EHDG_TILED_CH 1
#endif
// minimum resident blocks per SM asked of the compiler (instances with up
// to 28 face points per element)
#ifndef EHDG_TILED_MINB
#define EHDG_TILED_MINB 3
#endif
constexpr int kTW = EHDG_TILED_TW;
constexpr int kTS = EHDG_TILED_TS;
constexpr int kCH = EHDG_TILED_CH;
static_assert(kCH == 1 || kCH == 2 || kCH == 4, "FMA chains per row: 1, 2 or 4");
constexpr uint32_t kTileWaitLimit = 1u << 22; // mbarrier polls before giving up
constexpr int kTiledMaxBlocks = 4096;         // same bound as the other transport sweep

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

// device allocation recorded in the context (freed by ehdg_destroy)
cudaError_t dalloc_raw(Ctx& c, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) return e;
  c.allocs.push_back(*p);
  c.bytes += (int64_t)bytes;
  return cudaSuccess;
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// lane 0 only: start the copy of one operator row into a stage
__device__ __forceinline__ void issue_row(uint32_t mbar, uint32_t dst, const double* src,
                                          uint32_t bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// bounded wait for a phase of an mbarrier; true when it completed
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kTileWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
        " selp.u32 %0, 1, 0, w;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// bounded wait polled by every lane of a warp (each lane then sees the
// stage's data); the result is warp-uniform
__device__ __forceinline__ bool wait_phase_warp(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kTileWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
        " selp.u32 %0, 1, 0, w;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (__all_sync(0xffffffffu, done)) return true;
  }
  return false;
}

// Each warp owns an equal, contiguous range of the operator's rows (so every
// warp has the same work to within one row, whatever the tile boundaries) and
// runs on its own: no block barrier before the final residual reduction.
template <int F, int NQF>
__global__ void __launch_bounds__(32 * kTW, (F * NQF <= 28) ? EHDG_TILED_MINB : 1)
    k_sweep_tiled(const TiledParams p) {
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
  const int kk = p.it->k;                        // read before the last block advances it
  const int64_t tlen = (int64_t)NQF * nface;
  const double* src = p.uhat + (int64_t)(kk & 1) * tlen;
  double* dst = p.uhat + (int64_t)((kk + 1) & 1) * tlen;

  const int64_t nwarps = (int64_t)gridDim.x * kTW, gw = (int64_t)blockIdx.x * kTW + w;
  const int64_t J0 = p.total_rows * gw / nwarps, J1 = p.total_rows * (gw + 1) / nwarps;

  // producer: rows J0 .. J1-1 are contiguous in the operator, kTS ahead
  int64_t Jp = J0;
  for (int s = 0; s < kTS && Jp < J1; ++s, ++Jp)
    if (lane == 0)
      issue_row(saddr(&mbar[w][s]), saddr(stages + (size_t)s * NQ * 32), p.Hyt + Jp * NQ * 32,
                kRowBytes);

  double acc_res = 0.0;
  int64_t t = J0 < J1 ? p.warp_tile[gw] : p.ntiles;
  int j = J0 < J1 ? (int)(J0 - p.tile_row0[t]) : 0;
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
  if (J0 < J1 && t * 32 + lane < ne) {
    gy_n = p.Gy[(int64_t)j * ne + t * 32 + lane];
    rid_n = p.rowid[(int64_t)j * ne + t * 32 + lane];
  }
  int64_t J = J0;
  for (; J < J1; ++J) {
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
        for (int g = 0; g < NQF; ++g)
          u[f * NQF + g] = live ? src[(int64_t)g * nface + fid[f]] : 0.0;
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
      if (J + 1 < J1) load_tile(t);
    }
    if (J + 1 < J1 && t * 32 + lane < ne) {
      gy_n = p.Gy[(int64_t)j * ne + t * 32 + lane];
      rid_n = p.rowid[(int64_t)j * ne + t * 32 + lane];
    }

    const int st = (int)((J - J0) % kTS);
    if (!wait_phase_warp(saddr(&mbar[w][st]), (uint32_t)(((J - J0) / kTS) & 1))) {
      if (lane == 0) atomicExch(p.err, 1);
      break;
    }
    const double* Hs = stages + (size_t)st * NQ * 32;
    double a[kCH];
    a[0] = row_live ? gy : 0.0;
#pragma unroll
    for (int q = 1; q < kCH; ++q) a[q] = 0.0;
#pragma unroll
    for (int c = 0; c < NQ; ++c) a[c % kCH] = fma(Hs[c * 32 + lane], u[c], a[c % kCH]);
    double acc = a[0];
    if constexpr (kCH == 2) acc = a[0] + a[1];
    if constexpr (kCH == 4) acc = (a[0] + a[1]) + (a[2] + a[3]);
    __syncwarp();                                // every lane has read the stage
    if (Jp < J1) {
      if (lane == 0)
        issue_row(saddr(&mbar[w][st]), saddr(stages + (size_t)st * NQ * 32),
                  p.Hyt + Jp * NQ * 32, kRowBytes);
      ++Jp;
    }
    if (row_live) {
      const int f = rid / NQF, g = rid - f * NQF;
      int face = 0;
      double jfv = 0.0, uk = 0.0;
#pragma unroll
      for (int q = 0; q < F; ++q)
        if (q == f) {
          face = fid[q];
          jfv = jf[q];
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
  // copies still in flight (only after a wait gave up): wait for them, bounded
  for (int64_t Jw = J; Jw < Jp; ++Jw) {
    const int st = (int)((Jw - J0) % kTS);
    if (lane == 0) wait_phase(saddr(&mbar[w][st]), (uint32_t)(((Jw - J0) / kTS) & 1));
  }
  __syncwarp();
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

// Low-precision correction sweep of the mixed form (delta = R + S Hy delta,
// the correction equation of the FP64 trace fixed point), FP32 on the CUDA
// cores, with an FP32 copy of the tile-major operator. Same row ranges and
// warp starts as the FP64 sweep; rows are half as long, so each warp keeps
// kLS stages in the same shared memory. Owned points: out = R + row value;
// rows of points with beta.n = 0 go to Y32 for the finishing kernel.
constexpr int kLS = 2 * kTS;

struct LpTParams {
  int64_t nel, nface, ntiles, total_rows;
  const int32_t* warp_tile;
  const int32_t* tile_row0;
  const uint8_t* tile_nrows;
  const uint8_t* rowid;
  const uint8_t* nrows;
  const uint8_t* nup;
  const int32_t* elem_face;
  const float* Hyt32;           // tile-major rows, FP32
  const float* R;               // [Nqf][nface]
  const float* in;
  float* out;
  float* Y32;                   // [NQFS][nel]
  int* err;
};

template <int F, int NQF>
__global__ void __launch_bounds__(32 * kTW) k_sweep_lp_tiled(const LpTParams p) {
  constexpr int NQ = F * NQF;
  constexpr uint32_t kRowBytes = (uint32_t)NQ * 32u * 4u;
  extern __shared__ __align__(256) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar[kTW][kLS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* stages = reinterpret_cast<float*>(tsm) + (size_t)w * kLS * NQ * 32;
  if (lane == 0) {
    for (int s = 0; s < kLS; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[w][s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();

  const int64_t ne = p.nel, nface = p.nface;
  const int64_t nwarps = (int64_t)gridDim.x * kTW, gw = (int64_t)blockIdx.x * kTW + w;
  const int64_t J0 = p.total_rows * gw / nwarps, J1 = p.total_rows * (gw + 1) / nwarps;
  int64_t Jp = J0;
  for (int s = 0; s < kLS && Jp < J1; ++s, ++Jp)
    if (lane == 0)
      issue_row(saddr(&mbar[w][s]), saddr(stages + (size_t)s * NQ * 32),
                reinterpret_cast<const double*>(p.Hyt32 + Jp * NQ * 32), kRowBytes);

  int64_t t = J0 < J1 ? p.warp_tile[gw] : p.ntiles;
  int j = J0 < J1 ? (int)(J0 - p.tile_row0[t]) : 0;
  int nr_t = 0, nr_e = 0, nu_e = 0;
  int64_t e = 0;
  int fid[F];
  float d[NQ];
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
  bool fresh = true;
  int rid_n = (J0 < J1 && t * 32 + lane < ne) ? p.rowid[(int64_t)j * ne + t * 32 + lane] : 0;
  int64_t J = J0;
  for (; J < J1; ++J) {
    if (fresh) {
      e = t * 32 + lane;
      const bool live = e < ne;
      nr_t = nr_t_n;
      nr_e = nr_e_n;
      nu_e = nu_e_n;
#pragma unroll
      for (int f = 0; f < F; ++f) {
        fid[f] = fid_n[f];
#pragma unroll
        for (int g = 0; g < NQF; ++g)
          d[f * NQF + g] = live ? p.in[(int64_t)g * nface + fid[f]] : 0.f;
      }
      fresh = false;
    }
    const bool row_live = j < nr_e;
    const int rid = rid_n;
    const bool owned = row_live && j < nu_e;
    // the owned point and its R value, loaded before the FMA chain
    const int f0 = rid / NQF, g0 = rid - f0 * NQF;
    int face = 0;
#pragma unroll
    for (int q = 0; q < F; ++q)
      if (q == f0) face = fid[q];
    const int64_t pt = (int64_t)g0 * nface + face;
    const float rv = owned ? p.R[pt] : 0.f;
    if (++j == nr_t) {
      j = 0;
      do {
        ++t;
      } while (t < p.ntiles && p.tile_nrows[t] == 0);
      fresh = true;
      if (J + 1 < J1) load_tile(t);
    }
    if (J + 1 < J1 && t * 32 + lane < ne) rid_n = p.rowid[(int64_t)j * ne + t * 32 + lane];

    const int st = (int)((J - J0) % kLS);
    if (!wait_phase_warp(saddr(&mbar[w][st]), (uint32_t)(((J - J0) / kLS) & 1))) {
      if (lane == 0) atomicExch(p.err, 1);
      break;
    }
    const float* Hs = stages + (size_t)st * NQ * 32;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int c = 0; c < NQ; c += 2) {
      a0 = fmaf(Hs[c * 32 + lane], d[c], a0);
      if (c + 1 < NQ) a1 = fmaf(Hs[(c + 1) * 32 + lane], d[c + 1], a1);
    }
    const float acc = a0 + a1;
    __syncwarp();                                // every lane has read the stage
    if (Jp < J1) {
      if (lane == 0)
        issue_row(saddr(&mbar[w][st]), saddr(stages + (size_t)st * NQ * 32),
                  reinterpret_cast<const double*>(p.Hyt32 + Jp * NQ * 32), kRowBytes);
      ++Jp;
    }
    if (owned) {
      p.out[pt] = rv + acc;
    } else if (row_live) {
      p.Y32[(int64_t)rid * ne + e] = acc;
    }
  }
  for (int64_t Jw = J; Jw < Jp; ++Jw) {
    const int st = (int)((Jw - J0) % kLS);
    if (lane == 0) wait_phase(saddr(&mbar[w][st]), (uint32_t)(((Jw - J0) / kLS) & 1));
  }
  __syncwarp();
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

// FP32 rounding of an FP64 array
__global__ void k_round_f32(int64_t n, const double* src, float* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
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

// launch shape of one kernel instance: dynamic shared memory and a one-wave
// grid with at least four rows per warp
template <class K>
cudaError_t tiled_shape_of(K kern, int NQ, int64_t total_rows, int64_t ntiles, int* grid,
                           size_t* smem_out) {
  const size_t smem = sizeof(double) * (size_t)kTW * kTS * NQ * 32;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  int bpsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, kern, 32 * kTW, smem) != cudaSuccess ||
      bpsm < 1) {
    cudaGetLastError();
    bpsm = 1;
  }
  int64_t g = (int64_t)bpsm * device_sms();
  const int64_t by_rows = (total_rows + 4 * kTW - 1) / (4 * kTW);
  if (g > by_rows) g = by_rows;
  if (g > ntiles) g = ntiles;
  if (g > kTiledMaxBlocks) g = kTiledMaxBlocks;
  if (g < 1) g = 1;
  *grid = (int)g;
  *smem_out = smem;
  return cudaSuccess;
}

template <int F, int NQF>
cudaError_t tiled_config(int64_t total_rows, int64_t ntiles, int* grid, size_t* smem_out) {
  return tiled_shape_of(k_sweep_tiled<F, NQF>, F * NQF, total_rows, ntiles, grid, smem_out);
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
template <int F, int NQF>
cudaError_t lp_launch(const LpTParams& p, int grid, cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)kTW * kLS * F * NQF * 32;
  auto kern = k_sweep_lp_tiled<F, NQF>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<grid, 32 * kTW, smem, s>>>(p);
  return cudaGetLastError();
}

template <int F, int NQF>
cudaError_t tiled_launch(const TiledParams& p, int grid, size_t smem, cudaStream_t s) {
  k_sweep_tiled<F, NQF><<<grid, 32 * kTW, smem, s>>>(p);
  return cudaGetLastError();
}

struct TiledOps {
  cudaError_t (*config)(int64_t, int64_t, int*, size_t*);
  cudaError_t (*launch)(const TiledParams&, int, size_t, cudaStream_t);
  cudaError_t (*final_config)(int64_t, int64_t, int*, size_t*);
  cudaError_t (*final_launch)(const FinalTParams&, int, size_t, cudaStream_t);
  cudaError_t (*lp_launch)(const LpTParams&, int, cudaStream_t);
};

template <int F, int NQF>
constexpr TiledOps ops_of() {
  return TiledOps{&tiled_config<F, NQF>, &tiled_launch<F, NQF>, &final_config<F, NQF>,
                  &final_launch<F, NQF>, &lp_launch<F, NQF>};
}

// (faces, points per face) pairs with a kernel instance: quadrilaterals with
// 2..10 Gauss points per edge, hexahedra with 2x2 or 3x3 per face
bool tiled_ops(int F, int Nqf, TiledOps* out) {
  if (F == 4) {
    switch (Nqf) {
      case 2: *out = ops_of<4, 2>(); return true;
      case 3: *out = ops_of<4, 3>(); return true;
      case 4: *out = ops_of<4, 4>(); return true;
      case 5: *out = ops_of<4, 5>(); return true;
      case 6: *out = ops_of<4, 6>(); return true;
      case 7: *out = ops_of<4, 7>(); return true;
      case 8: *out = ops_of<4, 8>(); return true;
      case 9: *out = ops_of<4, 9>(); return true;
      case 10: *out = ops_of<4, 10>(); return true;
      default: return false;
    }
  }
  if (F == 6 && Nqf == 4) { *out = ops_of<6, 4>(); return true; }
  if (F == 6 && Nqf == 9) { *out = ops_of<6, 9>(); return true; }
  return false;
}

}  // namespace

bool tiled_supported(const Ctx& c) {
  TiledOps ops;
  return c.pde == EHDG_TRANSPORT && !c.shared_op && tiled_ops(c.F, c.Nqf, &ops);
}

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
  TiledOps ops;
  if (!tiled_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  if ((err = ops.config(rows, ntiles, &c.tiled_grid, &c.tiled_smem)) != cudaSuccess) return err;
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
    // FP32 copy of the tile-major sweep operator for the correction sweeps
    const int64_t n32 = rows * c.NQFS * 32;
    if ((err = dalloc_raw(c, (void**)&c.Hyt32, sizeof(float) * (size_t)std::max<int64_t>(n32, 1))) !=
        cudaSuccess)
      return err;
    k_round_f32<<<152 * 8, 256, 0, c.stream>>>(n32, c.Hyt, c.Hyt32);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

cudaError_t launch_lp_sweep_tiled(Ctx& c, const float* in, float* out) {
  LpTParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.ntiles = c.ntiles;
  p.total_rows = c.tile_rows;
  p.warp_tile = c.tiled_warp_tile;
  p.tile_row0 = c.tile_row0;
  p.tile_nrows = c.tile_nrows;
  p.rowid = c.rowid;
  p.nrows = c.nrows;
  p.nup = c.nup;
  p.elem_face = c.geo.elem_face;
  p.Hyt32 = c.Hyt32;
  p.R = c.R32;
  p.in = in;
  p.out = out;
  p.Y32 = c.Y32;
  p.err = c.tc_err;
  TiledOps ops;
  if (!tiled_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  return ops.lp_launch(p, c.tiled_grid, c.stream);
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
  TiledOps ops;
  if (!tiled_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  return ops.final_launch(p, c.ftiled_grid, c.ftiled_smem, c.stream);
}

cudaError_t launch_sweep_tiled(Ctx& c, int graph_mode, int* grid_out) {
  TiledParams p;
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
  TiledOps ops;
  if (!tiled_ops(c.F, c.Nqf, &ops)) return cudaErrorInvalidValue;
  *grid_out = c.tiled_grid;
  return ops.launch(p, c.tiled_grid, c.tiled_smem, c.stream);
}

}  // namespace ehdg
