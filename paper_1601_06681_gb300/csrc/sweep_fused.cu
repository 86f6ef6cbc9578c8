// Fused transport sweep: element solve + trace formula + FP64 residual in one
// kernel (Sec. 3, eqs. transportLocalk1 and transportLocale).
//
// For transport the trace formula picks, at every face point, the value of
// the upwind element (sgn(beta.n) = +-1), so the upwind element owns the
// point and writes uhat^{k+1} there itself; every point has exactly one owner.
// Points with beta.n = 0 (average of both sides) are finished by a small
// kernel over a precomputed list; inflow boundary points hold g in both
// ping-pong slots for the whole step. The owner also adds the point's share
// of ||uhat^{k+1} - uhat^k||^2, with uhat^k taken from the values it staged
// for its own solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "ehdg_internal.h"
#include "fused_tile.cuh"
#include "sweep_common.cuh"

namespace ehdg {

namespace {

constexpr int kFusedMaxBlocks = 4096;

struct FusedParams {
  int64_t nel, nface;
  int NQFS, Nqf, F, shared, n_rows, n_up;
  const int* rows;              // shared operator: rows, upwind ones first
  const uint8_t* rowid;         // per-element operator: [slot][nel], upwind slots first
  const uint8_t* nrows;
  const uint8_t* nup;
  const int32_t* elem_face;     // [F][nel]
  const double* face_jf;        // [nface]
  double fw[kMaxQ * kMaxQ];
  double* uhat;                 // [2][Nqf][nface]
  IterState* it;
  const double* Gy;
  const double* Hy;
  double* Y;                    // rows of tangential points, for the finishing kernel
  float* R_out;                 // mixed precision: F(uhat) - uhat at owned points (or null)
  double* partials;
  int final_here;               // 1: this kernel's last block finishes the residual
  double tol, res_scale;
  int max_iter;
  double* hist;
  int graph_mode;
  cudaGraphConditionalHandle handle;
};

// FT: row groups per 32-element tile (the block is 32 x FT threads); each row
// of an element is one thread's FMA chain whatever FT is, so the sweep's
// values do not depend on it (only the residual's summation order does).
template <int NQ, int FT>
__global__ void __launch_bounds__(32 * FT, 16 / FT)
    k_sweep_fused(const __grid_constant__ FusedParams p) {
  extern __shared__ double sm[];
  const int nq = NQ > 0 ? NQ : p.NQFS;
  const int lane = threadIdx.x, t = threadIdx.y;
  double* Hsh = sm;
  double* uh = sm + (p.shared ? nq * nq : 0);            // [nq][32]
  int* fid = reinterpret_cast<int*>(uh + nq * 32);        // [F][32]
  if (p.shared)
    for (int i = t * 32 + lane; i < nq * nq; i += 32 * FT) Hsh[i] = p.Hy[i];
  const int64_t ne = p.nel, nface = p.nface;
  const int kk = p.it->k;                                 // read before the last block advances it
  const int64_t tlen = (int64_t)p.Nqf * nface;
  const double* src = p.uhat + (int64_t)(kk & 1) * tlen;
  double* dst = p.uhat + (int64_t)((kk + 1) & 1) * tlen;
  const int64_t ntiles = (ne + 31) / 32;
  double acc_res = 0.0;
  if (p.shared) {
    // the tile body the batched loop runs too (same arithmetic)
    const FusedTileView v = {p.nel, p.nface, p.NQFS, p.Nqf, p.F, p.n_rows, p.n_up, p.rows,
                             p.elem_face, p.face_jf, p.fw, p.Gy, p.Y, p.R_out};
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      fused_tile_shared<NQ, FT>(v, Hsh, uh, fid, src, dst, tile, acc_res);
  } else
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e = tile * 32 + lane;
    __syncthreads();                                      // previous tile done with uh/fid
    if (e < ne) {
      for (int f = t; f < p.F; f += FT) fid[f * 32 + lane] = p.elem_face[f * ne + e];
    }
    __syncthreads();
    if (e < ne) {
      for (int i = t; i < nq; i += FT) {
        const int f = i / p.Nqf, g = i - f * p.Nqf;
        uh[i * 32 + lane] = src[g * nface + fid[f * 32 + lane]];
      }
    }
    __syncthreads();
    if (e < ne) {
      const int nr = p.shared ? p.n_rows : p.nrows[e];
      const int nu = p.shared ? p.n_up : p.nup[e];
      for (int j = t; j < nr; j += FT) {
        // two independent FMA chains (even and odd columns)
        double a0 = p.Gy[j * ne + e], a1 = 0.0;
        int r;
        if (p.shared) {
          r = p.rows[j];
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
        } else {
          r = p.rowid[j * ne + e];
          const double* Hr = p.Hy + (int64_t)j * nq * ne + e;
          if constexpr (NQ > 0) {
#pragma unroll 16
            for (int c = 0; c < NQ; c += 2) {
              a0 = fma(Hr[c * ne], uh[c * 32 + lane], a0);
              if (c + 1 < NQ) a1 = fma(Hr[(c + 1) * ne], uh[(c + 1) * 32 + lane], a1);
            }
          } else {
            for (int c = 0; c < nq; ++c) a0 = fma(Hr[c * ne], uh[c * 32 + lane], a0);
          }
        }
        const double acc = a0 + a1;
        if (j < nu) {
          const int f = r / p.Nqf, g = r - f * p.Nqf;
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
  }
  if (p.final_here) {
    finish_residual(acc_res, p.partials, blockIdx.x, gridDim.x, p.it, p.hist, p.max_iter, p.tol,
                    p.res_scale, p.graph_mode, p.handle, gridDim.x);
  } else {
    // partial sums only; the finishing kernel reduces them with its own
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

// Points with beta.n = 0: average of the two sides (eq. transportLocale with
// sgn = 0), and the final residual reduction over both kernels' partials.
struct TangentParams {
  int64_t nel, nface, n_tan;
  int Nqf, cn;
  const int32_t* tan_g;
  const int32_t* tan_face;
  const int32_t* face_elem;     // [2][nface]
  const int8_t* face_local;     // [2][nface]
  const double* face_jf;
  double fw[kMaxQ * kMaxQ];
  const double* gb;
  const double* gb_old;
  const double* Y;
  double* uhat;
  float* R_out;
  IterState* it;
  double* partials;             // [elem blocks + own blocks]
  int elem_blocks;
  double tol, res_scale;
  int max_iter;
  double* hist;
  int graph_mode;
  cudaGraphConditionalHandle handle;
};

__global__ void __launch_bounds__(256) k_tangent(const TangentParams p) {
  const int64_t nface = p.nface, ne = p.nel;
  const int kk = p.it->k;
  const int64_t tlen = (int64_t)p.Nqf * nface;
  const double* src = p.uhat + (int64_t)(kk & 1) * tlen;
  double* dst = p.uhat + (int64_t)((kk + 1) & 1) * tlen;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_tan;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = p.tan_g[i];
    const int64_t face = p.tan_face[i];
    const int em = p.face_elem[face], ep = p.face_elem[nface + face];
    const int fm = p.face_local[face], fpl = p.face_local[nface + face];
    const double ym = p.Y[(int64_t)(fm * p.Nqf + g) * ne + em];
    double yp;
    if (ep >= 0) {
      yp = p.Y[(int64_t)(fpl * p.Nqf + g) * ne + ep];
    } else {
      const int64_t t = (int64_t)g * nface + face;
      yp = p.cn ? 0.5 * (p.gb[t] + p.gb_old[t]) : p.gb[t];
    }
    const double v = 0.5 * (ym + yp);
    const int64_t t = (int64_t)g * nface + face;
    const double d = v - src[t];
    dst[t] = v;
    acc += p.face_jf[face] * p.fw[g] * d * d;
    if (p.R_out) p.R_out[t] = (float)d;
  }
  finish_residual(acc, p.partials, p.elem_blocks + blockIdx.x, gridDim.x, p.it, p.hist,
                  p.max_iter, p.tol, p.res_scale, p.graph_mode, p.handle,
                  p.elem_blocks + gridDim.x);
}

}  // namespace

int tangent_grid(int64_t n_tan) {
  int g = (int)((n_tan + 255) / 256);
  if (g > 152 * 4) g = 152 * 4;
  return g < 1 ? 1 : g;
}

int fused_grid(int64_t nel) {
  int64_t g = (nel + 31) / 32;
  if (g > kFusedMaxBlocks) g = kFusedMaxBlocks;
  return g < 1 ? 1 : (int)g;
}

void fill_face_weights(const Ctx& c, double* fw) {
  for (int g = 0; g < c.Nqf; ++g) {
    double w = 1.0;
    int rem = g;
    for (int t = 0; t < c.dim - 1; ++t) {
      w *= c.r1d.om[rem % c.q];
      rem /= c.q;
    }
    fw[g] = w;
  }
}

int device_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 152;
  }
  return nsm;
}

// Function attributes and occupancy are set or queried once per kernel and
// size, not per launch: they cost host time on every call (which also shows
// in the per-launch event timings of host-driven steps), the dynamic
// shared-memory limit is only ever raised (a lower limit would invalidate
// launches captured into graphs with a higher one), and the carveout is set
// once.
namespace {
std::mutex g_fn_mu;
std::map<std::pair<int, const void*>, size_t> g_fn_smem;
std::map<std::pair<int, const void*>, bool> g_fn_carve;
std::map<std::tuple<int, const void*, int, size_t>, int> g_fn_occ;
int cur_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}
}  // namespace

cudaError_t fn_smem(const void* fn, size_t bytes) {
  const auto key = std::make_pair(cur_device(), fn);
  std::lock_guard<std::mutex> lk(g_fn_mu);
  auto it = g_fn_smem.find(key);
  if (it != g_fn_smem.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g_fn_smem[key] = bytes;
  return e;
}

cudaError_t fn_carveout(const void* fn) {
  const auto key = std::make_pair(cur_device(), fn);
  std::lock_guard<std::mutex> lk(g_fn_mu);
  if (g_fn_carve.count(key)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) g_fn_carve[key] = true;
  return e;
}

// Resident blocks per SM from the kernel's registers and shared memory and the
// device's per-SM limits (registers allocated per warp in units of 256).
static int blocks_from_attrs(const void* fn, int threads, size_t smem) {
  cudaFuncAttributes fa;
  int dev = 0, regs_sm = 0, thr_sm = 0, smem_sm = 0, smem_rsv = 0, blk_sm = 0;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs > 0 ? fa.numRegs : 1) * 32 + 255) / 256 * 256;
  int b = blk_sm;
  b = std::min(b, (regs_sm / regs_warp) / warps);
  b = std::min(b, thr_sm / (warps * 32));
  const size_t per_block = smem + fa.sharedSizeBytes + (size_t)smem_rsv;
  if (per_block > 0) b = std::min<int>(b, (int)((size_t)smem_sm / per_block));
  return b;
}

int fn_blocks_from_attrs(const void* fn, int threads, size_t smem) {
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  const auto key = std::make_tuple(cur_device(), fn, threads, smem);
  std::lock_guard<std::mutex> lk(g_fn_mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const int b = blocks_from_attrs(fn, threads, smem);
  if (b > 0) cache[key] = b;
  return b;
}

int fn_blocks_per_sm(const void* fn, int threads, size_t smem) {
  const auto key = std::make_tuple(cur_device(), fn, threads, smem);
  std::lock_guard<std::mutex> lk(g_fn_mu);
  auto it = g_fn_occ.find(key);
  if (it != g_fn_occ.end()) return it->second;
  int bpsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, fn, threads, smem) != cudaSuccess ||
      bpsm < 1) {
    cudaGetLastError();
    return 1;                    // not cached: a later call may succeed
  }
  g_fn_occ[key] = bpsm;
  return bpsm;
}

// Persistent grid: one full wave of resident blocks (no partial last wave),
// capped by the number of 32-element tiles and by `cap`.
template <class K>
int one_wave_grid(K kernel, int threads, size_t smem, int64_t ntiles, int cap) {
  const int bpsm = fn_blocks_per_sm((const void*)kernel, threads, smem);
  int64_t g = (int64_t)bpsm * device_sms();
  if (g > ntiles) g = ntiles;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

template <int NQ, int FT>
static cudaError_t launch_fused_ft(const FusedParams& p, size_t smem, int64_t ntiles,
                                   cudaStream_t s, int* grid_out) {
  cudaError_t err = fn_smem((const void*)k_sweep_fused<NQ, FT>, smem);
  if (err != cudaSuccess) return err;
  const int grid = one_wave_grid(k_sweep_fused<NQ, FT>, 32 * FT, smem, ntiles, kFusedMaxBlocks);
  *grid_out = grid;
  k_sweep_fused<NQ, FT><<<grid, dim3(32, FT), smem, s>>>(p);
  return cudaGetLastError();
}

// The grid a launch of the fused sweep uses (one wave of resident blocks,
// capped by the tiles): the number of residual partials of the instance.
template <int NQ>
static int fused_grid_t(size_t smem, int64_t ntiles, int ft) {
  switch (ft) {
    case 2: return one_wave_grid(k_sweep_fused<NQ, 2>, 64, smem, ntiles, kFusedMaxBlocks);
    case 8: return one_wave_grid(k_sweep_fused<NQ, 8>, 256, smem, ntiles, kFusedMaxBlocks);
    default: return one_wave_grid(k_sweep_fused<NQ, 4>, 128, smem, ntiles, kFusedMaxBlocks);
  }
}

template <int NQ>
static cudaError_t launch_fused_t(const FusedParams& p, size_t smem, int64_t ntiles, int ft,
                                  cudaStream_t s, int* grid_out) {
  switch (ft) {
    case 2: return launch_fused_ft<NQ, 2>(p, smem, ntiles, s, grid_out);
    case 8: return launch_fused_ft<NQ, 8>(p, smem, ntiles, s, grid_out);
    default: return launch_fused_ft<NQ, 4>(p, smem, ntiles, s, grid_out);
  }
}

size_t fused_sweep_smem(const Ctx& c) {
  return sizeof(double) * ((c.shared_op ? (size_t)c.NQFS * c.NQFS : 0) + (size_t)c.NQFS * 32) +
         sizeof(int) * c.F * 32;
}

int fused_sweep_grid(const Ctx& c) {
  const size_t smem = fused_sweep_smem(c);
  const int64_t ntiles = (c.nel + 31) / 32;
  switch (c.NQFS) {
    case 8: return fused_grid_t<8>(smem, ntiles, c.sweep_ft);
    case 12: return fused_grid_t<12>(smem, ntiles, c.sweep_ft);
    case 16: return fused_grid_t<16>(smem, ntiles, c.sweep_ft);
    case 20: return fused_grid_t<20>(smem, ntiles, c.sweep_ft);
    case 24: return fused_grid_t<24>(smem, ntiles, c.sweep_ft);
    case 28: return fused_grid_t<28>(smem, ntiles, c.sweep_ft);
    case 36: return fused_grid_t<36>(smem, ntiles, c.sweep_ft);
    case 40: return fused_grid_t<40>(smem, ntiles, c.sweep_ft);
    case 54: return fused_grid_t<54>(smem, ntiles, c.sweep_ft);
    case 96: return fused_grid_t<96>(smem, ntiles, c.sweep_ft);
    default: return fused_grid_t<0>(smem, ntiles, c.sweep_ft);
  }
}

cudaError_t launch_sweep_fused(Ctx& c, int graph_mode) {
  FusedParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.NQFS = c.NQFS;
  p.Nqf = c.Nqf;
  p.F = c.F;
  p.shared = c.shared_op ? 1 : 0;
  p.n_rows = c.n_rows;
  p.n_up = c.n_up;
  p.rows = c.rows;
  p.rowid = c.rowid;
  p.nrows = c.nrows;
  p.nup = c.nup;
  p.elem_face = c.geo.elem_face;
  p.face_jf = c.geo.face_jf;
  fill_face_weights(c, p.fw);
  p.uhat = c.uhat;
  p.it = c.it;
  p.Gy = c.Gy;
  p.Hy = c.Hy;
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
  const size_t smem = fused_sweep_smem(c);
  const int64_t ntiles = (c.nel + 31) / 32;
  int grid = 1;
  cudaError_t err;
  if (c.use_ozaki) {
    err = launch_sweep_ozaki(c, graph_mode, &grid);
  } else if (c.Hyt) {
    err = launch_sweep_tiled(c, graph_mode, &grid);
  } else if (c.use_sf) {
    err = launch_sweep_sf(c, graph_mode, &grid);
  } else if (c.use_pe) {
    err = launch_sweep_pe(c, graph_mode, &grid);
  } else switch (c.NQFS) {
    case 8: err = launch_fused_t<8>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 12: err = launch_fused_t<12>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 16: err = launch_fused_t<16>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 20: err = launch_fused_t<20>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 24: err = launch_fused_t<24>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 28: err = launch_fused_t<28>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 36: err = launch_fused_t<36>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 40: err = launch_fused_t<40>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 54: err = launch_fused_t<54>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    case 96: err = launch_fused_t<96>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
    default: err = launch_fused_t<0>(p, smem, ntiles, c.sweep_ft, c.stream, &grid); break;
  }
  if (err != cudaSuccess || c.n_tan == 0) return err;
  TangentParams q;
  q.nel = c.nel;
  q.nface = c.nface;
  q.n_tan = c.n_tan;
  q.Nqf = c.Nqf;
  q.cn = (c.scheme == EHDG_CN) ? 1 : 0;
  q.tan_g = c.tan_g;
  q.tan_face = c.tan_face;
  q.face_elem = c.geo.face_elem;
  q.face_local = c.geo.face_local;
  q.face_jf = c.geo.face_jf;
  fill_face_weights(c, q.fw);
  q.gb = c.gb;
  q.gb_old = c.gb_old;
  q.Y = c.Y;
  q.uhat = c.uhat;
  q.R_out = c.mixed ? c.R32 : nullptr;
  q.it = c.it;
  q.partials = c.partials;
  q.elem_blocks = grid;
  q.tol = c.tol;
  q.res_scale = c.res_scale;
  q.max_iter = c.max_iter;
  q.hist = c.hist;
  q.graph_mode = graph_mode;
  q.handle = c.handle;
  k_tangent<<<tangent_grid(c.n_tan), 256, 0, c.stream>>>(q);
  return cudaGetLastError();
}

}  // namespace ehdg
