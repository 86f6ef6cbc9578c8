// Low-precision correction sweep on the 5th-generation tensor cores (tcgen05),
// for a local operator shared by every element (constant velocity on a
// uniform mesh): Ydelta = delta_loc Hy^T is a dense GEMM with
//   M = elements (128 per tile, one TMEM lane each), K = face points of an
//   element (NQFS, padded), N = sweep rows (upwind first, padded to 16),
// operands TF32 or BF16 in shared memory, FP32 accumulation in TMEM.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, adjacent core matrices along K 128 bytes
// apart (LBO) and 8-row groups (K bytes / 16) * 128 bytes apart (SBO).
// One thread issues the MMAs and commits them to an mbarrier; every wait on
// the mbarrier is bounded and records an error instead of hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "umma.cuh"

namespace ehdg {

namespace {

constexpr int kTcM = 128;
constexpr int kTcThreads = 256;                // two threads per element (tile row)
constexpr uint32_t kWaitLimit = 1u << 24;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

struct TcParams {
  int64_t nel, nface;
  int NQFS, Nqf, F, n_rows, n_up, owner_writes;
  int Kp, Np, ncols;            // padded K and N, TMEM columns
  int bf16;                     // 1: kind::f16 with BF16 operands, 0: kind::tf32
  uint32_t idesc;
  const int* rows;
  const int32_t* elem_face;
  const float* Hy32;            // [NQFS][NQFS] shared operator
  const float* R;
  const float* in;
  float* out;
  float* Y32;
  int* err;
};

// one 16-byte chunk (one row of one core matrix): 4 TF32 or 8 BF16 values
__device__ __forceinline__ void store_chunk(unsigned char* dst, const float* v, int per, int bf16) {
  if (bf16) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat16 lo = __float2bfloat16_rn(v[2 * q]);
      const __nv_bfloat16 hi = __float2bfloat16_rn(v[2 * q + 1]);
      w[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    *reinterpret_cast<uint4*>(dst) =
        make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
  }
  (void)per;
}

__device__ __forceinline__ void store_elem(unsigned char* base, int row, int k, int esize,
                                           uint32_t sbo, float v, int bf16) {
  const uint32_t off = kmajor_off(row, k * esize, sbo);
  if (bf16) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
  } else {
    *reinterpret_cast<uint32_t*>(base + off) = to_tf32(v);
  }
}

// A's half H (K range [H Kp/2, (H+1) Kp/2)) of one element, when the faces F_
// and face points NQF are compile-time constants: after unrolling, every face
// and point index below is a constant, so each value costs one load from a
// register face id plus a constant point offset.
template <int F_, int NQF, int BF16, int H>
__device__ __forceinline__ void tc_gather_fixed(unsigned char* As, uint32_t rowoff,
                                                const float* in, const int* fid, int row,
                                                int64_t nface, bool live) {
  constexpr int NQFS = F_ * NQF;
  constexpr int KSTEP = BF16 ? 16 : 8;                 // elements per 32-byte MMA K step
  constexpr int KP = (NQFS + KSTEP - 1) / KSTEP * KSTEP;
  constexpr int KHALF = KP / 2;
  constexpr int K0 = H * KHALF;
  constexpr int CH = BF16 ? 8 : 4;                     // values per 16-byte chunk
  constexpr int F0 = K0 / NQF;
  constexpr int NF = (K0 + KHALF - 1) / NQF - F0 + 1;  // faces this half touches
  static_assert(KHALF % CH == 0, "whole chunks per half");
  int fr[NF];
#pragma unroll
  for (int m = 0; m < NF; ++m) fr[m] = (live && F0 + m < F_) ? fid[(F0 + m) * kTcM + row] : 0;
#pragma unroll
  for (int c = 0; c < KHALF / CH; ++c) {
    float v[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int k = K0 + c * CH + q;
      const int f = k / NQF, g = k - (k / NQF) * NQF;
      v[q] = (live && k < NQFS) ? in[(int64_t)g * nface + fr[f - F0]] : 0.f;
    }
    store_chunk(As + rowoff + (uint32_t)((K0 + c * CH) / CH) * 128u, v, CH, BF16);
  }
}

// F_, NQF > 0: faces and face points per face known at compile time, with
// BF16 the operand format; F_ = NQF = 0: the general form (format from p.bf16).
template <int F_, int NQF, int BF16>
__global__ void __launch_bounds__(kTcThreads) k_sweep_tc(const TcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kTcM - 1), half = tid >> 7;   // tile row (element) and K / N half
  const int esize = p.bf16 ? 2 : 4;
  const uint32_t kbytes = (uint32_t)p.Kp * esize;
  const uint32_t sbo = kbytes * 8u;             // (K bytes / 16) core matrices of 128 B
  unsigned char* Bs = sm;                        // Np x Kp
  unsigned char* As = sm + (size_t)p.Np * kbytes; // 128 x Kp
  int* fid = reinterpret_cast<int*>(As + (size_t)kTcM * kbytes);   // [F][128]
  int* row_f = fid + p.F * kTcM;                                   // [Np] face of a row
  int* row_g = row_f + p.Np;                                       // [Np] point of a row
  for (int j = tid; j < p.Np; j += kTcThreads) {
    const int r = j < p.n_rows ? p.rows[j] : 0;
    row_f[j] = r / p.Nqf;
    row_g[j] = r - (r / p.Nqf) * p.Nqf;
  }

  // B = sweep rows of the shared operator, zero-padded
  for (int i = tid; i < p.Np * p.Kp; i += kTcThreads) {
    const int n = i / p.Kp, k = i - n * p.Kp;
    float v = 0.f;
    if (n < p.n_rows && k < p.NQFS) v = p.Hy32[p.rows[n] * p.NQFS + k];
    store_elem(Bs, n, k, esize, sbo, v, p.bf16);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(p.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;

  const int64_t ne = p.nel, nface = p.nface;
  const int64_t ntiles = (ne + kTcM - 1) / kTcM;
  uint32_t phase = 0;
  bool failed = false;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t e = tile * kTcM + row;
    // A = this tile's correction values at its elements' face points: each
    // element's K range is split between its two threads; face/point counters
    // advance incrementally and 16 loads are in flight per round
    __syncthreads();
    if (e < ne)
      for (int f = half; f < p.F; f += 2) fid[f * kTcM + row] = p.elem_face[f * ne + e];
    __syncthreads();
    if constexpr (NQF > 0) {
      const uint32_t rowoff = (uint32_t)(row >> 3) * sbo + (uint32_t)(row & 7) * 16u;
      if (half == 0)
        tc_gather_fixed<F_, NQF, BF16, 0>(As, rowoff, p.in, fid, row, nface, e < ne);
      else
        tc_gather_fixed<F_, NQF, BF16, 1>(As, rowoff, p.in, fid, row, nface, e < ne);
    } else {
      const uint32_t rowoff = (uint32_t)(row >> 3) * sbo + (uint32_t)(row & 7) * 16u;
      const int khalf = p.Kp / 2;                        // a multiple of the chunk size
      const int kbeg = half * khalf, kend = kbeg + khalf;
      int f = kbeg / p.Nqf, g = kbeg - (kbeg / p.Nqf) * p.Nqf;
      for (int k0 = kbeg; k0 < kend; k0 += 16) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float x = 0.f;
          if (e < ne && k0 + q < p.NQFS && k0 + q < kend) {
            x = p.in[g * nface + fid[f * kTcM + row]];
            if (++g == p.Nqf) {
              g = 0;
              ++f;
            }
          }
          v[q] = x;
        }
        if (p.bf16) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (k0 + 8 * h < kend)
              store_chunk(As + rowoff + (uint32_t)((k0 + 8 * h) / 8) * 128u, v + 8 * h, 8, 1);
        } else {
#pragma unroll
          for (int h = 0; h < 4; ++h)
            if (k0 + 4 * h < kend)
              store_chunk(As + rowoff + (uint32_t)((k0 + 4 * h) / 4) * 128u, v + 4 * h, 4, 0);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const int ksteps = (int)(kbytes / 32u);
      for (int s = 0; s < ksteps; ++s) {
        const uint64_t ad = umma_desc(a0 + 256u * s, 128u, sbo);
        const uint64_t bd = umma_desc(b0 + 256u * s, 128u, sbo);
        const uint32_t acc = s > 0 ? 1u : 0u;
        if (p.bf16) {
          asm volatile(
              "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tbase),
              "l"(ad), "l"(bd), "r"(p.idesc), "r"(acc));
        } else {
          asm volatile(
              "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n" ::"r"(tbase),
              "l"(ad), "l"(bd), "r"(p.idesc), "r"(acc));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar)));
    }
    // bounded wait for the MMAs: one thread polls the mbarrier, the others
    // wait at the block barrier (no issue slots burnt while the MMA runs)
    uint32_t ok = 1;
    if (tid == 0) {
      ok = 0;
      for (uint32_t it = 0; it < kWaitLimit; ++it) {
        asm volatile(
            "{\n .reg .pred w;\n mbarrier.try_wait.parity.shared::cta.b64 w, [%1], %2;\n"
            " selp.u32 %0, 1, 0, w;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(&mbar)), "r"(phase)
            : "memory");
        if (ok) break;
      }
    }
    // block-uniform outcome, so every thread takes the same path below
    if (__syncthreads_or(ok ? 0 : 1)) {
      if (tid == 0) atomicExch(p.err, 1);
      failed = true;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (its elements) and
      // the columns of its half of N, 8 at a time
      const int nhalf = p.Np / 2;
      const int cbeg = half * nhalf, cend = cbeg + nhalf;
      for (int c0 = cbeg; c0 < cend; c0 += 8) {
        uint32_t v[8];
        const uint32_t taddr = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (e < ne) {
          int64_t pt[8];
          float rv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = c0 + q;
            pt[q] = -1;
            rv[q] = 0.f;
            if (j < p.n_rows && p.owner_writes && j < p.n_up) {
              pt[q] = (int64_t)row_g[j] * nface + fid[row_f[j] * kTcM + row];
              rv[q] = p.R[pt[q]];
            }
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = c0 + q;
            if (j >= p.n_rows) break;
            const float acc = __uint_as_float(v[q]);
            if (pt[q] >= 0) {
              p.out[pt[q]] = rv[q] + acc;
            } else {
              p.Y32[(int64_t)(row_f[j] * p.Nqf + row_g[j]) * ne + e] = acc;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(p.ncols));
}

// The kernel of a face shape: quadrilaterals with 2..7 points per edge and
// hexahedra with 2x2, 3x3 or 4x4 points per face have a compile-time form.
using TcKernel = void (*)(const TcParams);
template <int F_, int NQF>
TcKernel tc_pick(int bf16) {
  return bf16 ? k_sweep_tc<F_, NQF, 1> : k_sweep_tc<F_, NQF, 0>;
}
TcKernel tc_kernel(int F, int Nqf, int bf16) {
  if (F == 4) {
    switch (Nqf) {
      case 2: return tc_pick<4, 2>(bf16);
      case 3: return tc_pick<4, 3>(bf16);
      case 4: return tc_pick<4, 4>(bf16);
      case 5: return tc_pick<4, 5>(bf16);
      case 6: return tc_pick<4, 6>(bf16);
      case 7: return tc_pick<4, 7>(bf16);
      default: break;
    }
  } else if (F == 6) {
    switch (Nqf) {
      case 4: return tc_pick<6, 4>(bf16);
      case 9: return tc_pick<6, 9>(bf16);
      case 16: return tc_pick<6, 16>(bf16);
      default: break;
    }
  }
  return k_sweep_tc<0, 0, 0>;
}

}  // namespace

bool tc_supported(const Ctx& c) {
  // one shared operator, N (rows) and K (face points) small enough for one MMA tile
  return c.shared_op && c.n_rows >= 1 && c.n_rows <= 256 && c.NQFS <= 256;
}

cudaError_t launch_lp_sweep_tc(Ctx& c, const float* in, float* out) {
  TcParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.NQFS = c.NQFS;
  p.Nqf = c.Nqf;
  p.F = c.F;
  p.n_rows = c.n_rows;
  p.n_up = c.n_up;
  p.owner_writes = (c.pde == EHDG_TRANSPORT) ? 1 : 0;
  p.bf16 = (c.precision == EHDG_MIXED_BF16) ? 1 : 0;
  const int kstep = p.bf16 ? 16 : 8;                // elements per 32-byte MMA K step
  p.Kp = (c.NQFS + kstep - 1) / kstep * kstep;
  p.Np = (c.n_rows + 15) / 16 * 16;
  if (p.Np < 16) p.Np = 16;
  int ncols = 32;
  while (ncols < p.Np) ncols *= 2;
  p.ncols = ncols;
  const uint32_t fmt = p.bf16 ? 1u : 2u;            // BF16 (kind::f16) or TF32
  p.idesc = umma_idesc(fmt, kTcM, p.Np);
  p.rows = c.rows;
  p.elem_face = c.geo.elem_face;
  p.Hy32 = c.Hy32;
  p.R = c.R32;
  p.in = in;
  p.out = out;
  p.Y32 = c.Y32;
  p.err = c.tc_err;
  const int esize = p.bf16 ? 2 : 4;
  const size_t smem = (size_t)(p.Np + kTcM) * p.Kp * esize +
                      sizeof(int) * ((size_t)c.F * kTcM + 2 * (size_t)p.Np) + 1024;
  void (*kern)(const TcParams) = tc_kernel(c.F, c.Nqf, p.bf16);
  cudaError_t err =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // favour shared memory over L1 so several tiles' blocks fit per SM
  err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  // resident blocks per SM: shared memory (227 KB per SM usable) and TMEM (512 columns)
  int bpsm = (int)((227 * 1024) / (smem + 1024));
  if (bpsm > 512 / ncols) bpsm = 512 / ncols;
  if (bpsm > 8) bpsm = 8;
  if (bpsm < 1) bpsm = 1;
  const int64_t ntiles = (c.nel + kTcM - 1) / kTcM;
  int64_t grid = (int64_t)bpsm * device_sms();
  if (grid > ntiles) grid = ntiles;
  kern<<<(int)grid, kTcThreads, smem, c.stream>>>(p);
  return cudaGetLastError();
}

}  // namespace ehdg
