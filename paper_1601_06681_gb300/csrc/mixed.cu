// Mixed-precision defect correction for the eHDG trace fixed point.
//
// The FP64 iteration is uhat <- F(uhat) = T(Gy + Hy uhat; g) (Algorithm 1
// with the element solve folded into Hy). Each outer step of the mixed form
// evaluates the FP64 residual R = F(uhat) - uhat in one FP64 sweep (which also
// applies the FP64 convergence test), then solves the correction equation
//     delta = R + S Hy delta        (S: the linear part of the trace formula)
// approximately with m low-precision eHDG sweeps started from delta = R, and
// sets uhat <- uhat + delta in FP64. The fixed point is the FP64 one (R = 0),
// so the result meets the FP64 stopping rule of the plain path.
//
// Low-precision operands: FP32 on the CUDA cores (precision MIXED_FP32), or
// TF32/BF16 on the tensor cores for a shared operator (tc_sweep.cu); the
// operator is kept as an FP32 copy of Hy in the sweep's slot layout.
#include <cuda_runtime.h>

#include "ehdg_internal.h"

namespace ehdg {

namespace {

constexpr int kLT = 4;   // row groups per 32-element tile

// ---------------------------------------------------------------------------
// transport: fused low-precision sweep, owner-writes
//   out[pt] = R[pt] + (Hy32 in_loc)[row of the upwind element at pt]
// ---------------------------------------------------------------------------
struct LpParams {
  int64_t nel, nface;
  int NQFS, Nqf, F, shared, n_rows, n_up;
  const int* rows;
  const uint8_t* rowid;
  const uint8_t* nrows;
  const uint8_t* nup;
  const int32_t* elem_face;
  const float* Hy32;            // shared [NQFS][NQFS] or per element [slot][NQFS][nel]
  const float* R;               // [Nqf][nface]
  const float* in;              // [Nqf][nface]
  float* out;                   // [Nqf][nface]
  float* Y32;                   // [NQFS][nel] tangential rows / all rows (shallow water)
  int owner_writes;             // transport: write out at owned points; else Y32 only
};

template <int NQ>
__global__ void __launch_bounds__(32 * kLT) k_sweep_lp(const LpParams p) {
  extern __shared__ float smf[];
  const int nq = NQ > 0 ? NQ : p.NQFS;
  const int lane = threadIdx.x, t = threadIdx.y;
  float* Hsh = smf;
  float* dl = smf + (p.shared ? nq * nq : 0);           // [nq][32]
  int* fid = reinterpret_cast<int*>(dl + nq * 32);       // [F][32]
  if (p.shared)
    for (int i = t * 32 + lane; i < nq * nq; i += 32 * kLT) Hsh[i] = p.Hy32[i];
  const int64_t ne = p.nel, nface = p.nface;
  const int64_t ntiles = (ne + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e = tile * 32 + lane;
    const bool live = e < ne;
    const int nr = live ? (p.shared ? p.n_rows : p.nrows[e]) : 0;
    const int nu = (live && p.owner_writes) ? (p.shared ? p.n_up : p.nup[e]) : 0;
    // per-element operator: fetch the first pass's two rows now, so their
    // latency overlaps the trace gather below (they do not depend on it)
    float h1[NQ > 0 ? NQ : 1], h2[NQ > 0 ? NQ : 1];
    if constexpr (NQ > 0) {
      if (!p.shared) {
        const int j = t, j2 = t + kLT;
        const float* H1 = p.Hy32 + (int64_t)j * NQ * ne + e;
        const float* H2 = p.Hy32 + (int64_t)j2 * NQ * ne + e;
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
          h1[c] = (j < nr) ? H1[c * ne] : 0.f;
          h2[c] = (j2 < nr) ? H2[c * ne] : 0.f;
        }
      }
    }
    __syncthreads();
    if (live)
      for (int f = t; f < p.F; f += kLT) fid[f * 32 + lane] = p.elem_face[f * ne + e];
    __syncthreads();
    if (live) {
      for (int i = t; i < nq; i += kLT) {
        const int f = i / p.Nqf, g = i - f * p.Nqf;
        dl[i * 32 + lane] = p.in[g * nface + fid[f * 32 + lane]];
      }
    }
    __syncthreads();
    if (!live) continue;
    // two rows per pass (j and j + kLT) so twice as many loads are in flight
    for (int j = t; j < nr; j += 2 * kLT) {
      const int j2 = j + kLT;
      const bool two = j2 < nr;
      float a = 0.f, b = 0.f;
      int r, r2;
      if (p.shared) {
        r = p.rows[j];
        r2 = two ? p.rows[j2] : r;
        const float* H1 = Hsh + r * nq;
        const float* H2 = Hsh + r2 * nq;
        for (int c = 0; c < nq; ++c) {
          const float d = dl[c * 32 + lane];
          a = fmaf(H1[c], d, a);
          b = fmaf(H2[c], d, b);
        }
      } else {
        r = p.rowid[j * ne + e];
        r2 = two ? p.rowid[j2 * ne + e] : r;
        if constexpr (NQ > 0) {
          if (j != t) {                       // later passes: fetch now
            const float* H1 = p.Hy32 + (int64_t)j * NQ * ne + e;
            const float* H2 = p.Hy32 + (int64_t)j2 * NQ * ne + e;
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
              h1[c] = H1[c * ne];
              h2[c] = two ? H2[c * ne] : 0.f;
            }
          }
#pragma unroll
          for (int c = 0; c < NQ; ++c) {
            const float d = dl[c * 32 + lane];
            a = fmaf(h1[c], d, a);
            b = fmaf(h2[c], d, b);
          }
        } else {
          const float* H1 = p.Hy32 + (int64_t)j * nq * ne + e;
          const float* H2 = p.Hy32 + (int64_t)(two ? j2 : j) * nq * ne + e;
          for (int c = 0; c < nq; ++c) {
            const float d = dl[c * 32 + lane];
            a = fmaf(H1[c * ne], d, a);
            b = fmaf(H2[c * ne], d, b);
          }
        }
      }
      for (int q = 0; q < (two ? 2 : 1); ++q) {
        const int jj = q ? j2 : j, rr = q ? r2 : r;
        const float acc = q ? b : a;
        if (jj < nu) {
          const int f = rr / p.Nqf, g = rr - f * p.Nqf;
          const int64_t pt = (int64_t)g * nface + fid[f * 32 + lane];
          p.out[pt] = p.R[pt] + acc;
        } else {
          p.Y32[(int64_t)rr * ne + e] = acc;
        }
      }
    }
  }
}

// transport, points with beta.n = 0: out = R + (Y32^- + Y32^+) / 2 (boundary: Y32^- / 2)
__global__ void k_tangent_lp(int64_t n_tan, int64_t nel, int64_t nface, int Nqf,
                             const int32_t* tan_g, const int32_t* tan_face,
                             const int32_t* face_elem, const int8_t* face_local, const float* Y32,
                             const float* R, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_tan;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int g = tan_g[i];
    const int64_t face = tan_face[i];
    const int em = face_elem[face], ep = face_elem[nface + face];
    const int fm = face_local[face], fp = face_local[nface + face];
    float v = Y32[(int64_t)(fm * Nqf + g) * nel + em];
    if (ep >= 0) v += Y32[(int64_t)(fp * Nqf + g) * nel + ep];
    const int64_t pt = (int64_t)g * nface + face;
    out[pt] = R[pt] + 0.5f * v;
  }
}

// shallow water: out = R + Y32^- + Y32^+ (wall: 2 Y32^-), the linear part of
// phihat = c^- + c^+
__global__ void k_face_lp_sw(int64_t nel, int64_t nface, int Nqf, const int32_t* face_elem,
                             const int8_t* face_local, const float* Y32, const float* R,
                             float* out) {
  const int g = blockIdx.y;
  for (int64_t face = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; face < nface;
       face += (int64_t)gridDim.x * blockDim.x) {
    const int em = face_elem[face], ep = face_elem[nface + face];
    const int fm = face_local[face], fp = face_local[nface + face];
    const float ym = Y32[(int64_t)(fm * Nqf + g) * nel + em];
    const float v = (ep >= 0) ? ym + Y32[(int64_t)(fp * Nqf + g) * nel + ep] : 2.0f * ym;
    const int64_t pt = (int64_t)g * nface + face;
    out[pt] = R[pt] + v;
  }
}

// uhat <- uhat + delta in FP64: slot K&1 = slot (K+1)&1 + delta, K = it->k
__global__ void k_apply(int64_t total, const IterState* it, double* uhat, const float* delta) {
  const int K = it->k;
  double* dst = uhat + (int64_t)(K & 1) * total;
  const double* src = uhat + (int64_t)((K + 1) & 1) * total;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[t] + (double)delta[t];
}

__global__ void k_to_f32(int64_t n, const double* src, float* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

template <int NQ>
cudaError_t launch_lp_t(const LpParams& p, size_t smem, int64_t ntiles, cudaStream_t s) {
  cudaError_t err = fn_smem((const void*)k_sweep_lp<NQ>, smem);
  if (err != cudaSuccess) return err;
  const int bpsm = fn_blocks_per_sm((const void*)k_sweep_lp<NQ>, 32 * kLT, smem);
  int64_t grid = (int64_t)bpsm * device_sms();     // one full wave, tiles strided
  if (grid > ntiles) grid = ntiles;
  k_sweep_lp<NQ><<<(int)grid, dim3(32, kLT), smem, s>>>(p);
  return cudaGetLastError();
}

int grid1d(int64_t n, int bs, int cap) {
  int64_t g = (n + bs - 1) / bs;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

// FP32 copy of the sweep operator (after the per-element row compaction)
cudaError_t launch_hy_to_f32(Ctx& c) {
  const int64_t n = (int64_t)c.NQFS * c.NQFS * (c.shared_op ? 1 : c.nel);
  k_to_f32<<<grid1d(n, 256, 152 * 32), 256, 0, c.stream>>>(n, c.Hy, c.Hy32);
  return cudaGetLastError();
}

// One low-precision sweep of the correction equation: in -> out. TF32/BF16
// run the element solve on the tensor cores (shared operator), FP32 on the
// CUDA cores.
cudaError_t launch_lp_sweep(Ctx& c, const float* in, float* out, bool fuse_apply) {
  if (c.Hyt32 || c.Hyt16) {
    cudaError_t err = launch_lp_sweep_tiled(c, in, out);
    if (err != cudaSuccess) return err;
    if (c.n_tan > 0) {
      k_tangent_lp<<<grid1d(c.n_tan, 256, 152 * 4), 256, 0, c.stream>>>(
          c.n_tan, c.nel, c.nface, c.Nqf, c.tan_g, c.tan_face, c.geo.face_elem,
          c.geo.face_local, c.Y32, c.R32, out);
      err = cudaGetLastError();
    }
    return err;
  }
  if (c.precision == EHDG_MIXED_TF32 || c.precision == EHDG_MIXED_BF16) {
    cudaError_t err = launch_lp_sweep_tc(c, in, out, fuse_apply);
    if (err != cudaSuccess) return err;
    if (c.pde == EHDG_TRANSPORT) {
      if (c.n_tan > 0) {
        k_tangent_lp<<<grid1d(c.n_tan, 256, 152 * 4), 256, 0, c.stream>>>(
            c.n_tan, c.nel, c.nface, c.Nqf, c.tan_g, c.tan_face, c.geo.face_elem,
            c.geo.face_local, c.Y32, c.R32, out);
        err = cudaGetLastError();
      }
    } else {
      const dim3 g2(grid1d(c.nface, 256, 2432 / c.Nqf), c.Nqf);
      k_face_lp_sw<<<g2, 256, 0, c.stream>>>(c.nel, c.nface, c.Nqf, c.geo.face_elem,
                                             c.geo.face_local, c.Y32, c.R32, out);
      err = cudaGetLastError();
    }
    return err;
  }
  if (c.use_pe) return launch_lp_sweep_pe(c, in, out);   // FP32, one thread per element
  LpParams p;
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
  p.Hy32 = c.Hy32;
  p.R = c.R32;
  p.in = in;
  p.out = out;
  p.Y32 = c.Y32;
  p.owner_writes = (c.pde == EHDG_TRANSPORT) ? 1 : 0;
  const size_t smem = sizeof(float) * ((p.shared ? (size_t)c.NQFS * c.NQFS : 0) +
                                       (size_t)c.NQFS * 32) + sizeof(int) * c.F * 32;
  const int64_t ntiles = (c.nel + 31) / 32;
  cudaError_t err;
  switch (c.NQFS) {
    case 8: err = launch_lp_t<8>(p, smem, ntiles, c.stream); break;
    case 12: err = launch_lp_t<12>(p, smem, ntiles, c.stream); break;
    case 16: err = launch_lp_t<16>(p, smem, ntiles, c.stream); break;
    case 20: err = launch_lp_t<20>(p, smem, ntiles, c.stream); break;
    case 24: err = launch_lp_t<24>(p, smem, ntiles, c.stream); break;
    case 28: err = launch_lp_t<28>(p, smem, ntiles, c.stream); break;
    case 36: err = launch_lp_t<36>(p, smem, ntiles, c.stream); break;
    case 40: err = launch_lp_t<40>(p, smem, ntiles, c.stream); break;
    case 54: err = launch_lp_t<54>(p, smem, ntiles, c.stream); break;
    case 96: err = launch_lp_t<96>(p, smem, ntiles, c.stream); break;
    default: err = launch_lp_t<0>(p, smem, ntiles, c.stream); break;
  }
  if (err != cudaSuccess) return err;
  if (c.pde == EHDG_TRANSPORT) {
    if (c.n_tan > 0) {
      k_tangent_lp<<<grid1d(c.n_tan, 256, 152 * 4), 256, 0, c.stream>>>(
          c.n_tan, c.nel, c.nface, c.Nqf, c.tan_g, c.tan_face, c.geo.face_elem,
          c.geo.face_local, c.Y32, c.R32, out);
      err = cudaGetLastError();
    }
  } else {
    const dim3 g2(grid1d(c.nface, 256, 2432 / c.Nqf), c.Nqf);
    k_face_lp_sw<<<g2, 256, 0, c.stream>>>(c.nel, c.nface, c.Nqf, c.geo.face_elem,
                                           c.geo.face_local, c.Y32, c.R32, out);
    err = cudaGetLastError();
  }
  return err;
}

cudaError_t launch_apply(Ctx& c, const float* delta) {
  const int64_t total = (int64_t)c.Nqf * c.nface;
  k_apply<<<grid1d(total, 256, 152 * 16), 256, 0, c.stream>>>(total, c.it, c.uhat, delta);
  return cudaGetLastError();
}

// Kernels of one low-precision sweep (the element kernel plus the trace
// kernel of tangential points or of shallow water).
int lp_sweep_launches(const Ctx& c) {
  return 1 + ((c.pde == EHDG_TRANSPORT) ? (c.n_tan > 0 ? 1 : 0) : 1);
}

// Output buffer of inner sweep j (the sweeps ping-pong between two buffers;
// sweep 0 reads R).
float* correction_out(Ctx& c, int j) { return c.d32 + (int64_t)(j & 1) * c.Nqf * c.nface; }

// The m inner sweeps and the FP64 update (made by the last inner sweep where
// tc_apply_fusable).
cudaError_t launch_correction(Ctx& c) {
  const float* in = c.R32;
  const bool fuse = tc_apply_fusable(c);
  for (int j = 0; j < c.inner_sweeps; ++j) {
    float* out = correction_out(c, j);
    cudaError_t e = launch_lp_sweep(c, in, out, fuse && j == c.inner_sweeps - 1);
    if (e != cudaSuccess) return e;
    in = out;
  }
  return fuse ? cudaSuccess : launch_apply(c, in);
}

}  // namespace ehdg
