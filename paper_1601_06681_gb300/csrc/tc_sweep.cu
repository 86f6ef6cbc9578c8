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
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ehdg_internal.h"
#include "tc_fx_tile.cuh"
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

// The general form: any face shape and row set (format from p.bf16).
__global__ void __launch_bounds__(kTcThreads) k_sweep_tc(const TcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
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
    {
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

// ---------------------------------------------------------------------------
// Fixed-shape form. Faces F_ and points per face NQF are compile-time
// constants, and the sweep rows are whole faces (a constant velocity: every
// point of a face is upwind, or every point tangential), listed face by face.
// Per tile, each thread loads its element's face ids (the next tile's are
// prefetched), gathers its half of the K range with 32-bit point indices and
// loads the residual R at its owned points before the MMA; the epilogue then
// only reads TMEM, adds and stores. The operator rows come rounded, in the
// shared-memory image, from setup. The MMAs (operands, K steps, descriptors)
// are those of the general form, so both give the same values bit for bit.

template <int F_, int NQF, int BF16, int TPE, bool APPLY>
__device__ __forceinline__ void fx_sweep(const TcFxParams& p) {
  using S = FxShape<F_, NQF, BF16, TPE>;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kTcM - 1), part = tid >> 7;
  unsigned char* Bs = sm;                                   // Np x Kp
  unsigned char* As = sm + (size_t)p.Np * S::KBYTES;        // 128 x Kp
  {
    const int n16 = (int)((uint32_t)p.Np * S::KBYTES / 16u);
    for (int i = tid; i < n16; i += S::THREADS) reinterpret_cast<uint4*>(Bs)[i] = p.img[i];
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
  const int64_t ne = p.nel;
  const int64_t ntiles = (ne + kTcM - 1) / kTcM;
  uint32_t phase = 0;
  bool failed = false;
  // face ids of this block's first tile; each tile prefetches the next one's
  int fn[F_];
  {
    const int64_t e = (int64_t)blockIdx.x * kTcM + row;
#pragma unroll
    for (int f = 0; f < F_; ++f) fn[f] = e < ne ? p.elem_face[f * ne + e] : 0;
  }
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    int fid[F_];
#pragma unroll
    for (int f = 0; f < F_; ++f) fid[f] = fn[f];
    const int64_t e2 = (tile + gridDim.x) * kTcM + row;
#pragma unroll
    for (int f = 0; f < F_; ++f) fn[f] = e2 < ne ? p.elem_face[f * ne + e2] : 0;
    // parts are warp-uniform (128 threads each)
    if (part == 0) {
      fx_tile<F_, NQF, BF16, TPE, 0, APPLY>(p, As, Bs, &mbar, tbase, phase, failed, tile, fid);
    } else if constexpr (TPE == 2) {
      fx_tile<F_, NQF, BF16, TPE, 1, APPLY>(p, As, Bs, &mbar, tbase, phase, failed, tile, fid);
    } else {
      if (part == 1)
        fx_tile<F_, NQF, BF16, TPE, 1, APPLY>(p, As, Bs, &mbar, tbase, phase, failed, tile, fid);
      else if (part == 2)
        fx_tile<F_, NQF, BF16, TPE, 2, APPLY>(p, As, Bs, &mbar, tbase, phase, failed, tile, fid);
      else
        fx_tile<F_, NQF, BF16, TPE, 3, APPLY>(p, As, Bs, &mbar, tbase, phase, failed, tile, fid);
    }
    // every thread's TMEM reads of this tile precede the next tile's MMA
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(p.ncols));
}

template <int F_, int NQF, int BF16, int TPE>
__global__ void __launch_bounds__(128 * TPE)
    k_sweep_tc_fx(const __grid_constant__ TcFxParams p) {
  fx_sweep<F_, NQF, BF16, TPE, false>(p);
}

// the last inner sweep, which also makes the FP64 update (its own kernel:
// the update's loads raise its registers, not the plain form's; held to
// three blocks per SM it spilled and ran slower, measured at 64^3)
template <int F_, int NQF, int BF16, int TPE>
__global__ void __launch_bounds__(128 * TPE)
    k_sweep_tc_fx_apply(const __grid_constant__ TcFxParams p) {
  fx_sweep<F_, NQF, BF16, TPE, true>(p);
}

struct FxKernel {
  void (*fn)(const TcFxParams) = nullptr;
  int threads = 0;
};
// TPE = WANT where each part's K range is whole 16-byte chunks, else 2
constexpr int fx_tpe(int F_, int NQF, int BF16, int WANT) {
  const int kstep = BF16 ? 16 : 8, ch = BF16 ? 8 : 4;
  const int kp = (F_ * NQF + kstep - 1) / kstep * kstep;
  return ((kp / WANT) % ch == 0 && NQF >= WANT) ? WANT : 2;
}
template <int F_, int NQF, int TPE>
FxKernel fx_pick_kernel(int bf16, bool apply) {
  constexpr int T0 = fx_tpe(F_, NQF, 0, TPE), T1 = fx_tpe(F_, NQF, 1, TPE);
  FxKernel k;
  if (apply)
    k.fn = bf16 ? k_sweep_tc_fx_apply<F_, NQF, 1, T1> : k_sweep_tc_fx_apply<F_, NQF, 0, T0>;
  else
    k.fn = bf16 ? k_sweep_tc_fx<F_, NQF, 1, T1> : k_sweep_tc_fx<F_, NQF, 0, T0>;
  k.threads = 128 * (bf16 ? T1 : T0);
  return k;
}
// quadrilaterals with 2..7 points per edge, hexahedra with 2x2, 3x3, 4x4 per
// face; two threads per element (four measured slower at 64^3, p = 3: one
// block of 512 threads per SM at 64 registers against three of 256)
FxKernel fx_kernel(int F, int Nqf, int bf16, bool apply = false) {
  if (F == 4) {
    switch (Nqf) {
      case 2: return fx_pick_kernel<4, 2, 2>(bf16, apply);
      case 3: return fx_pick_kernel<4, 3, 2>(bf16, apply);
      case 4: return fx_pick_kernel<4, 4, 2>(bf16, apply);
      case 5: return fx_pick_kernel<4, 5, 2>(bf16, apply);
      case 6: return fx_pick_kernel<4, 6, 2>(bf16, apply);
      case 7: return fx_pick_kernel<4, 7, 2>(bf16, apply);
      default: break;
    }
  } else if (F == 6) {
    switch (Nqf) {
      case 4: return fx_pick_kernel<6, 4, 2>(bf16, apply);
      case 9: return fx_pick_kernel<6, 9, 2>(bf16, apply);
      case 16: return fx_pick_kernel<6, 16, 2>(bf16, apply);
      default: break;
    }
  }
  return FxKernel{};
}

// Setup: the sweep rows of the shared operator rounded to TF32 / BF16 in the
// K-major image both forms stage (zero padding to Np x Kp).
__global__ void k_tc_image(const float* Hy32, const int* rows, int n_rows, int NQFS, int Np,
                           int Kp, int bf16, unsigned char* img) {
  const int esize = bf16 ? 2 : 4;
  const uint32_t sbo = (uint32_t)Kp * esize * 8u;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Np * Kp; i += gridDim.x * blockDim.x) {
    const int n = i / Kp, k = i - n * Kp;
    float v = 0.f;
    if (n < n_rows && k < NQFS) v = Hy32[rows[n] * NQFS + k];
    store_elem(img, n, k, esize, sbo, v, bf16);
  }
}

struct TcShape {
  int bf16, Kp, Np, ncols;
  uint32_t idesc;
  size_t smem;
};

TcShape tc_shape(const Ctx& c) {
  TcShape t;
  t.bf16 = (c.precision == EHDG_MIXED_BF16) ? 1 : 0;
  const int kstep = t.bf16 ? 16 : 8;                // elements per 32-byte MMA K step
  t.Kp = (c.NQFS + kstep - 1) / kstep * kstep;
  t.Np = (c.n_rows + 15) / 16 * 16;
  if (t.Np < 16) t.Np = 16;
  int ncols = 32;
  while (ncols < t.Np) ncols *= 2;
  t.ncols = ncols;
  const uint32_t fmt = t.bf16 ? 1u : 2u;            // BF16 (kind::f16) or TF32
  t.idesc = umma_idesc(fmt, kTcM, t.Np);
  const int esize = t.bf16 ? 2 : 4;
  t.smem = (size_t)(t.Np + kTcM) * t.Kp * esize +
           sizeof(int) * ((size_t)c.F * kTcM + 2 * (size_t)t.Np) + 1024;
  return t;
}

// resident blocks per SM: shared memory (227 KB per SM usable) and TMEM (512 columns)
int64_t tc_grid(const Ctx& c, const TcShape& t, size_t smem) {
  int bpsm = (int)((227 * 1024) / (smem + 1024));
  if (bpsm > 512 / t.ncols) bpsm = 512 / t.ncols;
  if (bpsm > 8) bpsm = 8;
  if (bpsm < 1) bpsm = 1;
  const int64_t ntiles = (c.nel + kTcM - 1) / kTcM;
  int64_t grid = (int64_t)bpsm * device_sms();
  return grid > ntiles ? ntiles : grid;
}

}  // namespace

bool tc_supported(const Ctx& c) {
  // one shared operator, N (rows) and K (face points) small enough for one MMA tile
  return c.shared_op && c.n_rows >= 1 && c.n_rows <= 256 && c.NQFS <= 256;
}

cudaError_t build_tc_image(Ctx& c) {
  if (!tc_supported(c) ||
      (c.precision != EHDG_MIXED_TF32 && c.precision != EHDG_MIXED_BF16))
    return cudaSuccess;
  const TcShape t = tc_shape(c);
  const size_t bytes = (size_t)t.Np * t.Kp * (t.bf16 ? 2 : 4);
  void* img = nullptr;
  cudaError_t err = dalloc_raw(c, &img, bytes);
  if (err != cudaSuccess) return err;
  k_tc_image<<<(t.Np * t.Kp + 255) / 256, 256, 0, c.stream>>>(c.Hy32, c.rows, c.n_rows, c.NQFS,
                                                              t.Np, t.Kp, t.bf16,
                                                              static_cast<unsigned char*>(img));
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  c.tc_img = img;
  // the fixed-shape form: a compile-time face shape, whole faces as rows (in
  // face order, points ascending), 32-bit point and value indices
  c.tc_fx = false;
  if (!fx_kernel(c.F, c.Nqf, 0).fn || c.n_rows % c.Nqf != 0 || c.n_up % c.Nqf != 0) return cudaSuccess;
  if ((int64_t)c.Nqf * c.nface >= (1ll << 31) || (int64_t)c.NQFS * c.nel >= (1ll << 31))
    return cudaSuccess;
  const int n_rf = c.n_rows / c.Nqf;
  if (n_rf > 6 || (int)c.rows_host.size() != c.n_rows) return cudaSuccess;
  const int n_up_f = (c.pde == EHDG_TRANSPORT) ? c.n_up / c.Nqf : 0;
  if (n_up_f > c.F / 2) return cudaSuccess;
  for (int i = 0; i < n_rf; ++i) {
    const int s = c.rows_host[i * c.Nqf] / c.Nqf;
    for (int g = 0; g < c.Nqf; ++g)
      if (c.rows_host[i * c.Nqf + g] != s * c.Nqf + g) return cudaSuccess;
    c.tc_rfs[i] = s;
  }
  c.tc_nrf = n_rf;
  c.tc_nupf = n_up_f;
  c.tc_fx = true;
  return cudaSuccess;
}

bool tc_apply_fusable(const Ctx& c) {
  return c.tc_fx && c.tc_img && c.pde == EHDG_TRANSPORT && c.n_tan == 0 &&
         (c.precision == EHDG_MIXED_TF32 || c.precision == EHDG_MIXED_BF16);
}

cudaError_t launch_lp_sweep_tc(Ctx& c, const float* in, float* out, bool fuse_apply) {
  const TcShape t = tc_shape(c);
  if (c.tc_fx && c.tc_img) {
    TcFxParams q;
    q.nel = c.nel;
    q.nface = (uint32_t)c.nface;
    q.n_rf = c.tc_nrf;
    q.n_up_f = c.tc_nupf;
    for (int i = 0; i < 6; ++i) q.rfs[i] = c.tc_rfs[i];
    q.Np = t.Np;
    q.ncols = t.ncols;
    q.idesc = t.idesc;
    q.elem_face = c.geo.elem_face;
    q.img = static_cast<const uint4*>(c.tc_img);
    q.R = c.R32;
    q.in = in;
    q.out = out;
    q.Y32 = c.Y32;
    q.err = c.tc_err;
    q.apply_uhat = fuse_apply ? c.uhat : nullptr;
    q.apply_k = fuse_apply ? &c.it->k : nullptr;
    q.apply_total = (int64_t)c.Nqf * c.nface;
    const size_t smem = (size_t)(t.Np + kTcM) * t.Kp * (t.bf16 ? 2 : 4) + 1024;
    const FxKernel kern = fx_kernel(c.F, c.Nqf, t.bf16, fuse_apply);
    cudaError_t err = fn_smem((const void*)kern.fn, smem);
    if (err != cudaSuccess) return err;
    // favour shared memory over L1 so several tiles' blocks fit per SM
    err = fn_carveout((const void*)kern.fn);
    if (err != cudaSuccess) return err;
    // one wave of resident blocks (registers, shared memory; TMEM columns)
    int bpsm = std::max(fn_blocks_per_sm((const void*)kern.fn, kern.threads, smem),
                        fn_blocks_from_attrs((const void*)kern.fn, kern.threads, smem));
    if (bpsm > 512 / t.ncols) bpsm = 512 / t.ncols;
    const int64_t ntiles = (c.nel + kTcM - 1) / kTcM;
    int64_t grid = (int64_t)bpsm * device_sms();
    if (grid > ntiles) grid = ntiles;
    kern.fn<<<(int)grid, kern.threads, smem, c.stream>>>(q);
    return cudaGetLastError();
  }
  TcParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.NQFS = c.NQFS;
  p.Nqf = c.Nqf;
  p.F = c.F;
  p.n_rows = c.n_rows;
  p.n_up = c.n_up;
  p.owner_writes = (c.pde == EHDG_TRANSPORT) ? 1 : 0;
  p.bf16 = t.bf16;
  p.Kp = t.Kp;
  p.Np = t.Np;
  p.ncols = t.ncols;
  p.idesc = t.idesc;
  p.rows = c.rows;
  p.elem_face = c.geo.elem_face;
  p.Hy32 = c.Hy32;
  p.R = c.R32;
  p.in = in;
  p.out = out;
  p.Y32 = c.Y32;
  p.err = c.tc_err;
  cudaError_t err = fn_smem((const void*)k_sweep_tc, t.smem);
  if (err != cudaSuccess) return err;
  err = fn_carveout((const void*)k_sweep_tc);
  if (err != cudaSuccess) return err;
  k_sweep_tc<<<(int)tc_grid(c, t, t.smem), kTcThreads, t.smem, c.stream>>>(p);
  return cudaGetLastError();
}

}  // namespace ehdg
