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

constexpr int kTW = 2;                        // warps per block (independent)
constexpr int kTS = 3;                        // stages per warp
constexpr uint32_t kTileWaitLimit = 1u << 22; // mbarrier polls before giving up
constexpr int kTiledMaxBlocks = 4096;         // same bound as the other transport sweep

struct TiledParams {
  int64_t nel, nface, ntiles, total_rows;
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

// The tile holding global row J of the tile-major operator: the last tile
// whose first row is <= J (tiles without rows share their successor's first
// row, so the tile found has J among its rows).
__device__ __forceinline__ int64_t tile_of_row(const int32_t* row0, int64_t ntiles, int64_t J) {
  int64_t lo = 0, hi = ntiles - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)row0[mid] <= J) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Each warp owns an equal, contiguous range of the operator's rows (so every
// warp has the same work to within one row, whatever the tile boundaries) and
// runs on its own: no block barrier before the final residual reduction.
template <int F, int NQF>
__global__ void __launch_bounds__(32 * kTW) k_sweep_tiled(const TiledParams p) {
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
  int64_t t = J0 < J1 ? tile_of_row(p.tile_row0, p.ntiles, J0) : 0;
  int j = J0 < J1 ? (int)(J0 - p.tile_row0[t]) : 0;
  int nr_t = 0, nr_e = 0, nu_e = 0;
  int64_t e = 0;
  int fid[F];
  double jf[F], u[NQ];
  bool fresh = true;                             // tile t not gathered yet
  int64_t J = J0;
  for (; J < J1; ++J) {
    if (fresh) {
      // the element's faces, their Jacobians and uhat^k at its face points
      e = t * 32 + lane;
      const bool live = e < ne;
      nr_t = p.tile_nrows[t];
#pragma unroll
      for (int f = 0; f < F; ++f) fid[f] = live ? p.elem_face[(int64_t)f * ne + e] : 0;
#pragma unroll
      for (int f = 0; f < F; ++f) {
        jf[f] = live ? p.face_jf[fid[f]] : 0.0;
#pragma unroll
        for (int g = 0; g < NQF; ++g)
          u[f * NQF + g] = live ? src[(int64_t)g * nface + fid[f]] : 0.0;
      }
      nr_e = live ? p.nrows[e] : 0;
      nu_e = live ? p.nup[e] : 0;
      fresh = false;
    }
    // issued early, used after the FMA chain
    const bool row_live = j < nr_e;
    const double gy = row_live ? p.Gy[(int64_t)j * ne + e] : 0.0;
    const int rid = row_live ? p.rowid[(int64_t)j * ne + e] : 0;

    const int st = (int)((J - J0) % kTS);
    const uint32_t par = (uint32_t)(((J - J0) / kTS) & 1);
    bool ok = false;
    for (uint32_t it = 0; it < kTileWaitLimit; ++it) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
          " selp.u32 %0, 1, 0, w;\n}\n"
          : "=r"(done)
          : "r"(saddr(&mbar[w][st])), "r"(par)
          : "memory");
      if (__all_sync(0xffffffffu, done)) {
        ok = true;
        break;
      }
    }
    if (!ok) {
      if (lane == 0) atomicExch(p.err, 1);
      break;
    }
    const double* Hs = stages + (size_t)st * NQ * 32;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int c = 0; c < NQ; c += 4) {
      a0 = fma(Hs[c * 32 + lane], u[c], a0);
      if (c + 1 < NQ) a1 = fma(Hs[(c + 1) * 32 + lane], u[c + 1], a1);
      if (c + 2 < NQ) a2 = fma(Hs[(c + 2) * 32 + lane], u[c + 2], a2);
      if (c + 3 < NQ) a3 = fma(Hs[(c + 3) * 32 + lane], u[c + 3], a3);
    }
    const double acc = gy + ((a0 + a1) + (a2 + a3));
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
      if (j < nu_e) {
        const int64_t pt = (int64_t)g * nface + face;
        dst[pt] = acc;
        const double d = acc - uk;
        acc_res += jfv * p.fw[g] * d * d;
        if (p.R_out) p.R_out[pt] = (float)d;
      } else {
        p.Y[(int64_t)rid * ne + e] = acc;
      }
    }
    if (++j == nr_t) {                           // next tile with rows
      j = 0;
      do {
        ++t;
      } while (t < p.ntiles && p.tile_nrows[t] == 0);
      fresh = true;
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
cudaError_t launch_tiled_t(const TiledParams& p, int* grid_out, cudaStream_t s) {
  constexpr int NQ = F * NQF;
  const size_t smem = sizeof(double) * (size_t)kTW * kTS * NQ * 32;
  auto kern = k_sweep_tiled<F, NQF>;
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
  const int64_t by_rows = (p.total_rows + 4 * kTW - 1) / (4 * kTW);   // >= 4 rows per warp
  if (g > by_rows) g = by_rows;
  if (g > p.ntiles) g = p.ntiles;
  if (g > kTiledMaxBlocks) g = kTiledMaxBlocks;
  if (g < 1) g = 1;
  *grid_out = (int)g;
  kern<<<(int)g, 32 * kTW, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

// (faces, points per face) pairs with a kernel instance: quadrilaterals with
// 2..10 Gauss points per edge, hexahedra with 2x2 or 3x3 per face
static bool tiled_shape(int F, int Nqf) {
  if (F == 4) return Nqf >= 2 && Nqf <= 10;
  if (F == 6) return Nqf == 4 || Nqf == 9;
  return false;
}

bool tiled_supported(const Ctx& c) {
  return c.pde == EHDG_TRANSPORT && !c.shared_op && tiled_shape(c.F, c.Nqf);
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
  int grid = (int)std::min<int64_t>(ntiles, 152 * 16);
  k_tile_hy<<<grid < 1 ? 1 : grid, 256, 0, c.stream>>>(c.nel, c.NQFS, ntiles, c.tile_row0,
                                                       c.tile_nrows, c.nrows, c.Hy, c.Hyt);
  return cudaGetLastError();
}

cudaError_t launch_sweep_tiled(Ctx& c, int graph_mode, int* grid_out) {
  TiledParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.ntiles = c.ntiles;
  p.total_rows = c.tile_rows;
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
  if (c.F == 4) {
    switch (c.Nqf) {
      case 2: return launch_tiled_t<4, 2>(p, grid_out, c.stream);
      case 3: return launch_tiled_t<4, 3>(p, grid_out, c.stream);
      case 4: return launch_tiled_t<4, 4>(p, grid_out, c.stream);
      case 5: return launch_tiled_t<4, 5>(p, grid_out, c.stream);
      case 6: return launch_tiled_t<4, 6>(p, grid_out, c.stream);
      case 7: return launch_tiled_t<4, 7>(p, grid_out, c.stream);
      case 8: return launch_tiled_t<4, 8>(p, grid_out, c.stream);
      case 9: return launch_tiled_t<4, 9>(p, grid_out, c.stream);
      case 10: return launch_tiled_t<4, 10>(p, grid_out, c.stream);
      default: break;
    }
  } else if (c.F == 6) {
    if (c.Nqf == 4) return launch_tiled_t<6, 4>(p, grid_out, c.stream);
    if (c.Nqf == 9) return launch_tiled_t<6, 9>(p, grid_out, c.stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ehdg
