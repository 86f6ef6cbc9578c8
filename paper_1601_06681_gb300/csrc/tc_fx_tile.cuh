// Fixed-shape tile body of the tensor-core correction sweep (tcgen05), shared
// by the single-problem sweep and the batched loop: one 128-element tile of
// delta_out = R + delta_in Hy^T at the sweep rows, with the element's faces
// F_ and points per face NQF compile-time constants and the rows whole faces
// (upwind, owned faces first). TPE threads per element each gather a part of
// the K range into registers (all loads first), round it to TF32 / BF16 into
// the K-major A operand, and load R at their owned points; one thread issues
// the MMAs into the TMEM accumulator and commits to an mbarrier whose wait is
// bounded; the epilogue reads TMEM, adds R and stores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "umma.cuh"

namespace ehdg {

constexpr int kFxM = 128;                       // elements per tile (MMA M)
constexpr uint32_t kFxWaitLimit = 1u << 24;     // mbarrier polls before giving up

__device__ __forceinline__ uint32_t fx_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

struct TcFxParams {
  int64_t nel;
  uint32_t nface;
  int n_rf, n_up_f;             // row faces; leading ones the element owns (owner writes)
  int rfs[6];                   // local face of each row face
  int Np, ncols;
  uint32_t idesc;
  const int32_t* elem_face;     // [F][nel]
  const uint4* img;             // Np x Kp operator image (K-major, no swizzle)
  const float* R;
  const float* in;
  float* out;
  float* Y32;
  int* err;
  // the APPLY form (the last inner sweep of a transport step without
  // beta.n = 0 points): instead of storing the correction, apply it in FP64
  // at the owned points, uhat slot K&1 = slot (K+1)&1 + delta with
  // K = *apply_k (the FP64 update; points no element owns keep equal slots)
  double* apply_uhat;           // [2][apply_total] trace ping-pong pair
  const int* apply_k;
  int64_t apply_total;
};

template <int F_>
__device__ __forceinline__ int fx_pick(const int (&fid)[F_], int s) {
  int r = fid[0];
#pragma unroll
  for (int k = 1; k < F_; ++k) r = (s == k) ? fid[k] : r;
  return r;
}

// Compile-time shape of the fixed form: TPE threads per element (tile row),
// thread part q gathering K range [q KP/TPE, (q+1) KP/TPE) and owning points
// [q NQF/TPE, (q+1) NQF/TPE) of every row face in the epilogue (the last part
// takes the remainder).
template <int F_, int NQF, int BF16, int TPE>
struct FxShape {
  static constexpr int NQFS = F_ * NQF;
  static constexpr int KSTEP = BF16 ? 16 : 8;          // elements per 32-byte MMA K step
  static constexpr int KP = (NQFS + KSTEP - 1) / KSTEP * KSTEP;
  static constexpr uint32_t KBYTES = KP * (BF16 ? 2 : 4);
  static constexpr uint32_t SBO = KBYTES * 8u;
  static constexpr int CH = BF16 ? 8 : 4;              // values per 16-byte chunk
  static constexpr int KQ = KP / TPE;                  // K values a part gathers
  static constexpr int GQ = NQF / TPE;                 // epilogue points of parts 0..TPE-2
  static constexpr int GL = NQF - (TPE - 1) * GQ;      // ... and of the last part
  static constexpr int NUP = F_ / 2;                   // at most one outflow face per axis
  static constexpr int THREADS = 128 * TPE;
  static_assert(KQ % CH == 0, "whole chunks per part");
  static_assert(GQ >= 1, "every part owns points");
};

// GN consecutive accumulator columns of the warp's 32 lanes: one x8 load when
// GN = 8 at an 8-aligned column, else one x1 load per column
template <int GN, bool WIDE>
__device__ __forceinline__ void fx_tmem_ld(uint32_t taddr, uint32_t (&v)[GN]) {
  if constexpr (WIDE) {
    static_assert(GN == 8, "x8 load");
    tmem_ld8(taddr, v);
  } else {
#pragma unroll
    for (int q = 0; q < GN; ++q)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                   : "=r"(v[q])
                   : "r"(taddr + (uint32_t)q));
  }
}

// Thread part Q of element `row`: gathers its K range into registers (all
// loads first), rounds and stores it into A; loads R at its owned points;
// after the MMA, writes its points of every row face.
template <int F_, int NQF, int BF16, int TPE, int Q, bool APPLY = false>
__device__ __forceinline__ void fx_tile(const TcFxParams& p, unsigned char* As, unsigned char* Bs,
                                        uint64_t* mbar, uint32_t tbase, uint32_t& phase,
                                        bool& failed, int64_t tile, const int (&fid)[F_]) {
  using S = FxShape<F_, NQF, BF16, TPE>;
  constexpr int G0 = Q * S::GQ;                        // first point of this part
  constexpr int GN = (Q == TPE - 1) ? S::GL : S::GQ;   // points of this part
  constexpr bool WIDE = GN == 8 && (G0 % 8) == 0;
  constexpr int NUP = S::NUP;
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kFxM - 1);
  const int64_t ne = p.nel;
  const int64_t e = tile * kFxM + row;
  const bool live = e < ne;
  const uint32_t nface = p.nface;
  // every load of the tile first: R at the owned points, then the K range
  float rv[NUP][GN];
  int fo[NUP];
#pragma unroll
  for (int i = 0; i < NUP; ++i) {
    fo[i] = fx_pick<F_>(fid, p.rfs[i]);
#pragma unroll
    for (int q = 0; q < GN; ++q)
      rv[i][q] = i < p.n_up_f ? __ldg(p.R + ((uint32_t)(G0 + q) * nface + (uint32_t)fo[i])) : 0.f;
  }
  float v[S::KQ];
#pragma unroll
  for (int j = 0; j < S::KQ; ++j) {
    const int k = Q * S::KQ + j;
    const int f = k / NQF, g = k - (k / NQF) * NQF;
    v[j] = k < S::NQFS ? __ldg(p.in + ((uint32_t)g * nface + (uint32_t)fid[f < F_ ? f : 0])) : 0.f;
  }
  unsigned char* Arow = As + (uint32_t)(row >> 3) * S::SBO + (uint32_t)(row & 7) * 16u;
#pragma unroll
  for (int c = 0; c < S::KQ / S::CH; ++c) {
    unsigned char* dst = Arow + (uint32_t)(Q * S::KQ / S::CH + c) * 128u;
    const float* w = v + c * S::CH;
    if constexpr (BF16) {
      uint32_t u[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(w[2 * h], w[2 * h + 1]);
        u[h] = *reinterpret_cast<const uint32_t*>(&b);
      }
      *reinterpret_cast<uint4*>(dst) = make_uint4(u[0], u[1], u[2], u[3]);
    } else {
      *reinterpret_cast<uint4*>(dst) =
          make_uint4(fx_tf32(w[0]), fx_tf32(w[1]), fx_tf32(w[2]), fx_tf32(w[3]));
    }
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
    for (int s = 0; s < (int)(S::KBYTES / 32u); ++s) {
      const uint64_t ad = umma_desc(a0 + 256u * s, 128u, S::SBO);
      const uint64_t bd = umma_desc(b0 + 256u * s, 128u, S::SBO);
      const uint32_t acc = s > 0 ? 1u : 0u;
      if constexpr (BF16) {
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
            smem_u32(mbar)));
  }
  uint32_t ok = 1;
  if (tid == 0) ok = mbar_wait_bounded(mbar, phase, kFxWaitLimit) ? 1u : 0u;
  if (__syncthreads_or(ok ? 0 : 1)) {
    if (tid == 0) atomicExch(p.err, 1);
    failed = true;
    return;
  }
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tl = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)G0;
  const double* asrc = nullptr;
  double* adst = nullptr;
  if constexpr (APPLY) {
    const int K = *p.apply_k;
    adst = p.apply_uhat + (int64_t)(K & 1) * p.apply_total;
    asrc = p.apply_uhat + (int64_t)((K + 1) & 1) * p.apply_total;
  }
  // owned row faces: the new correction at the element's outflow points
#pragma unroll
  for (int i = 0; i < NUP; ++i) {
    if (i >= p.n_up_f) break;
    double sv[GN];   // APPLY: the update's FP64 trace values, loaded before the TMEM read
    if (APPLY && live) {
#pragma unroll
      for (int q = 0; q < GN; ++q) sv[q] = asrc[(uint32_t)(G0 + q) * nface + (uint32_t)fo[i]];
    }
    uint32_t a[GN];
    fx_tmem_ld<GN, WIDE>(tl + (uint32_t)(i * NQF), a);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (live) {
#pragma unroll
      for (int q = 0; q < GN; ++q) {
        const uint32_t pt = (uint32_t)(G0 + q) * nface + (uint32_t)fo[i];
        const float d = rv[i][q] + __uint_as_float(a[q]);
        if constexpr (APPLY)
          adst[pt] = sv[q] + (double)d;
        else
          p.out[pt] = d;
      }
    }
  }
  // the other row faces (tangential points; every face for shallow water)
  for (int i = p.n_up_f; i < p.n_rf; ++i) {
    uint32_t a[GN];
    fx_tmem_ld<GN, WIDE>(tl + (uint32_t)(i * NQF), a);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (live) {
      const int sl = p.rfs[i];
#pragma unroll
      for (int q = 0; q < GN; ++q)
        p.Y32[(int64_t)(sl * NQF + G0 + q) * ne + e] = __uint_as_float(a[q]);
    }
  }
}

}  // namespace ehdg
