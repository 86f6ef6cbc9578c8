// FP64-accurate transport sweep on the BF16 tensor cores (Ozaki splitting),
// for a local operator shared by every element (constant velocity, uniform
// mesh). The same kernel, in two more modes, forms the other two shared-
// operator products of an implicit step: the reconstruction u = G + H uhat
// and the step's right-hand side G = P w (Sec. 3, the local solve).
//
// Per eHDG iteration (Algorithm 1, Sec. 3) and element e, every sweep row n
// (a face point r_n of e) needs y = sum_j Hy[r_n][j] uhat_e[j]: the local
// solve (eq. transportLocalk1) evaluated at the face points, with Hy the
// face-point rows of A^{-1} B. The owner of the point then writes
// uhat^{k+1} = Gy + y (eq. transportLocale, upwind selection) and adds its
// share of the FP64 residual ||uhat^{k+1} - uhat^k||_{L2(E_h)}.
//
// Over all elements the products are one GEMM, M = elements, N = rows,
// K = face points. Here it runs as exact integer arithmetic:
//  - each element's traces go to fixed point against the element's largest
//    exponent E, X_j = round(|uhat_j| 2^(1071 - E)) < 2^49 + 1, and each
//    operator row against its own largest exponent, Y_nj;
//  - the signed X and Y are written in base 128 with seven digits,
//    X = x_0 2^42 + sum_{i>=1} x_i 2^(42 - 7 i): x_0 = floor(X / 2^42) in
//    [-128, 128] carries the sign and x_1..x_6 are in [0, 127], all exact in
//    BF16;
//  - tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation) sums the digit
//    products of level L = i + l into one TMEM accumulator per level,
//    L = 0..7. Every partial sum is an integer of magnitude below 2^24
//    (7 * K * 128 * 128 with K <= 144), so the FP32 accumulation is exact;
//  - the epilogue recombines the levels in 64-bit integers and builds the
//    double from its bits, then adds Gy and forms the residual in FP64.
// Rounding X and Y costs at most 2^-49 of the element's (row's) largest
// magnitude per operand; the dropped levels L >= 8 cost below 2^-51 of
// max|uhat_e| max|Hy_n| per product.
//
// Shared-memory operands use the K-major layout without swizzle. B holds the
// seven digit slices of the sweep rows stacked along N, LS rows each (the
// rows padded to a multiple of 32, zero beyond the sweep rows), and stays
// resident; level L's accumulator sits at TMEM column L * LS. So one MMA of
// A slice i against B slices l0 .. l0 + nl - 1 (N = nl * LS <= 256) feeds
// levels i + l0 .. i + l0 + nl - 1 at once, and each A slice is read from
// shared memory two or three times instead of seven. A (one digit slice of
// the tile's 128 elements) is double-buffered so that the digits of slice
// i + 1 are written while the MMAs of slice i run. One thread issues the
// MMAs and commits each slice to an mbarrier; every wait is bounded and
// records an error instead of hanging.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ehdg_internal.h"
#include "sweep_common.cuh"
#include "umma.cuh"

namespace ehdg {

namespace {

constexpr int kOzM = 128;                  // elements per tile (TMEM lanes)
constexpr int kOzDigits = 7;               // 7-bit digits per operand: 49-bit fixed point
constexpr int kOzLevels = 8;               // digit-product levels kept, L = i + l <= 7
constexpr uint32_t kOzWait = 1u << 24;     // mbarrier polls before giving up

// kOzSweep: one transport eHDG iteration (owner writes, residual);
// kOzElem: Y = Gy + Hy uhat at every sweep row (the shallow-water element
// apply; the trace kernel forms the trace and the residual); kOzFinal:
// u = G + H uhat; kOzStep: G = P w.
enum OzMode { kOzSweep = 0, kOzFinal = 1, kOzStep = 2, kOzElem = 3 };

struct OzParams {
  int64_t nel, nface;
  int NQFS, Nqf, F, n_rows, n_up;   // n_rows: output rows (sweep rows, or the n element nodes)
  int n_in;                     // step: entries of w (the n element nodes)
  int Np, LS, ncols;            // rows padded to 16, TMEM columns per level, allocated columns
  const int* rows;              // sweep rows (face points), upwind first
  const int32_t* elem_face;     // [F][nel]
  const double* face_jf;        // [nface]
  double fw[kMaxQ * kMaxQ];
  const uint4* Bimg;            // [kOzDigits * LS x KP] BF16 digits, K-major image
  const int* Fb;                // [LS] largest biased exponent of each row
  double* uhat;                 // [2][Nqf][nface]
  IterState* it;
  const double* Gy;             // [row][nel]
  double* Y;                    // [point][nel] rows of tangential points
  float* R_out;                 // mixed precision: F(uhat) - uhat at owned points (or null)
  // reconstruction: u = G + H uhat (cn: 2 (G + H uhat) - u); step: G = P w,
  // w = ucoef u + f (force_avg: (f + f_old) / 2)
  const double* G;
  double* u;
  double* Gout;
  const double* force;
  const double* force_old;
  double ucoef;
  int cn, have_force, force_avg;
  double* partials;
  int final_here;
  double tol, res_scale;
  int max_iter;
  double* hist;
  int graph_mode;
  cudaGraphConditionalHandle handle;
  int* err;
};

// Signed fixed point of x against biased exponent E >= that of x:
// round(x 2^(1071 - E)), of magnitude <= 2^49. Zeros and subnormals give 0
// (below the fixed point's resolution).
__host__ __device__ __forceinline__ int64_t oz_fixed(uint64_t bits, int E) {
  const int be = (int)((bits >> 52) & 0x7FF);
  if (be == 0) return 0;
  const int sh = E - be + 4;
  if (sh >= 54) return 0;
  const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int64_t a = (int64_t)((mant + (1ull << (sh - 1))) >> sh);
  return (bits >> 63) ? -a : a;
}

// Base-128 digit i of a signed fixed-point value as BF16 bits (exact):
// i = 0 is floor(X / 2^42) in [-128, 128], i >= 1 is in [0, 127].
template <int I>
__device__ __forceinline__ uint32_t oz_digit_bf16(int64_t X) {
  if (I == 0) {
    const int d = (int)(X >> 42);
    // 1.5 * 2^23 + d as float bits, minus 1.5 * 2^23: exactly d
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return __float_as_uint(f) >> 16;
  } else {
    const uint32_t d = (uint32_t)(X >> (42 - 7 * I)) & 127u;
    const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
    return __float_as_uint(f) >> 16;
  }
}

// T * 2^(sc - 1023) as a double, from the bits (|T| < 2^62; truncated to
// 53 bits; 0 below the normal range).
__device__ __forceinline__ double oz_to_double(int64_t T, int sc) {
  if (T == 0) return 0.0;
  const uint64_t s = (uint64_t)(T >> 63);
  const uint64_t a = ((uint64_t)T ^ s) - s;
  const int lz = __clzll((long long)a);
  const int be = 63 - lz + sc;
  if (be <= 0) return 0.0;
  if (be >= 2047) return __longlong_as_double((long long)((s << 63) | (0x7FFull << 52)));
  const uint64_t m = (a << lz) >> 11;
  return __longlong_as_double(
      (long long)((s << 63) | ((uint64_t)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void oz_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar)));
}

// Setup: digit slices and row exponents of the shared operator's sweep rows,
// one warp per padded row n < LS; digit l of row n is row l * LS + n of the
// stacked K-major image.
template <int I>
__device__ __forceinline__ void oz_put_digit(unsigned short* img, int LS, int KP, int n, int j,
                                             int64_t Yv) {
  const size_t off = kmajor_off(I * LS + n, 2 * j, 16u * (uint32_t)KP);
  img[off / 2] = (unsigned short)oz_digit_bf16<I>(Yv);
}

__global__ void k_oz_split_rows(const double* M, int ld, const int* rows, int n_rows, int K,
                                int LS, int KP, unsigned short* img, int* Fb) {
  const int n = blockIdx.x, lane = threadIdx.x;
  const double* Mr = M + (int64_t)(n < n_rows ? (rows ? rows[n] : n) : 0) * ld;
  int emax = 0;
  if (n < n_rows)
    for (int j = lane; j < K; j += 32) {
      const uint64_t b = (uint64_t)__double_as_longlong(Mr[j]);
      emax = max(emax, (int)((b >> 52) & 0x7FF));
    }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (lane == 0) Fb[n] = emax;
  for (int j = lane; j < KP; j += 32) {
    uint64_t bits = 0;
    if (n < n_rows && j < K) bits = (uint64_t)__double_as_longlong(Mr[j]);
    const int64_t Yv = oz_fixed(bits, emax);
    oz_put_digit<0>(img, LS, KP, n, j, Yv);
    oz_put_digit<1>(img, LS, KP, n, j, Yv);
    oz_put_digit<2>(img, LS, KP, n, j, Yv);
    oz_put_digit<3>(img, LS, KP, n, j, Yv);
    oz_put_digit<4>(img, LS, KP, n, j, Yv);
    oz_put_digit<5>(img, LS, KP, n, j, Yv);
    oz_put_digit<6>(img, LS, KP, n, j, Yv);
  }
}

// Per-CTA state of the sweep kernel that the slice steps share.
struct OzCta {
  unsigned char* As;            // [2][128 x KP] A digit buffers
  uint64_t* empty;              // [2] MMAs of the buffer's slice done (tcgen05.commit)
  uint64_t* full;               // [2] every thread's digits of the buffer's slice written
  uint64_t adesc[2];            // descriptors of the two A buffers (K step 0)
  uint64_t bdesc;               // descriptor of the stacked B slices (K step 0, slice 0)
  uint32_t bslice;              // descriptor address units (16 B) of one B slice
  uint32_t tbase;
  uint32_t idesc_n0;            // instruction descriptor without its N field
  uint32_t ph_empty[2], ph_full[2];
  bool ok;                      // every bounded wait of this thread succeeded
};

// Digit slice I of the tile. A thread waits until the buffer's previous slice
// (I - 2) has been consumed by the tensor cores, writes its digits and
// arrives on the buffer's "full" barrier; thread 0 then waits for every
// thread's digits and issues the MMAs of every level I + l <= 7, committed to
// the buffer's "empty" barrier. No block-wide barrier: writers run up to one
// slice ahead of the tensor cores.
template <int KP, int TPE, int I>
__device__ __forceinline__ void oz_slice(OzCta& t, const int64_t* X, uint32_t rowoff, uint32_t kc0,
                                         int LS, int tid) {
  constexpr int KH = KP / TPE;
  constexpr uint32_t ABYTES = (uint32_t)kOzM * KP * 2u;
  if (I >= 2) {
    t.ok = mbar_wait_bounded(&t.empty[I & 1], t.ph_empty[I & 1], kOzWait) && t.ok;
    t.ph_empty[I & 1] ^= 1u;
  }
  unsigned char* Ab = t.As + (I & 1) * ABYTES;
#pragma unroll
  for (int c8 = 0; c8 < KH / 8; ++c8) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = oz_digit_bf16<I>(X[c8 * 8 + 2 * q]) | (oz_digit_bf16<I>(X[c8 * 8 + 2 * q + 1]) << 16);
    *reinterpret_cast<uint4*>(Ab + rowoff + (kc0 + (uint32_t)c8) * 128u) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&t.full[I & 1]))
               : "memory");
  if (tid == 0) {
    const bool got = mbar_wait_bounded(&t.full[I & 1], t.ph_full[I & 1], kOzWait);
    t.ph_full[I & 1] ^= 1u;
    t.ok = got && t.ok;
    if (got) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // groups (first B slice, slices) of levels I .. 7, each N = slices * LS
      // <= 256; a group whose levels start their accumulators here (slice 0,
      // and level 7 at slice 1) holds no level that is already accumulating
      constexpr int ng = I == 1 ? 3 : (I <= 3 ? 2 : 1);
      constexpr int g0[3] = {0, 4, I == 1 ? 6 : 0};
      constexpr int gn[3] = {I <= 3 ? 4 : (I == 4 ? 4 : (I == 5 ? 3 : 2)),
                             I == 0 ? 3 : (I == 1 ? 2 : (I == 2 ? 2 : 1)), 1};
#pragma unroll
      for (int gi = 0; gi < ng; ++gi) {
        const bool first = I == 0 || (I == 1 && gi == 2);
        const uint32_t d = t.tbase + (uint32_t)((I + g0[gi]) * LS);
        const uint32_t idesc = t.idesc_n0 | ((uint32_t)((gn[gi] * LS) >> 3) << 17);
        const uint64_t b0 = t.bdesc + (uint64_t)(g0[gi] * t.bslice);
#pragma unroll
        for (int s = 0; s < KP / 16; ++s)
          oz_mma(d, t.adesc[I & 1] + 16u * s, b0 + 16u * s, idesc, (first && s == 0) ? 0u : 1u);
      }
    }
    // committed even without MMAs, so that no waiter is left hanging
    oz_commit(&t.empty[I & 1]);
  }
}

// This thread's KH traces of element e (raw FP64 bits); part PART of the
// element's face points when the face-point count NQF is known at compile
// time, so that every face and point index is a constant.
template <int KP, int NQF, int TPE, int PART>
__device__ __forceinline__ void oz_gather_part(int64_t* X, const double* src, const int* fid,
                                               int row, int64_t nface, int NQFS, bool live) {
  constexpr int KH = KP / TPE;
#pragma unroll
  for (int q = 0; q < KH; ++q) {
    const int k = PART * KH + q;
    const int f = k / NQF, g = k - f * NQF;
    X[q] = (live && k < NQFS)
               ? __double_as_longlong(src[(int64_t)g * nface + fid[f * kOzM + row]])
               : 0;
  }
}

template <int KP, int NQF, int TPE>
__device__ __forceinline__ void oz_gather(int64_t* X, const double* src, const int* fid, int row,
                                          int part, int64_t nface, int NQFS, int Nqf, bool live) {
  constexpr int KH = KP / TPE;
  if constexpr (NQF > 0) {
    if (part == 0) oz_gather_part<KP, NQF, TPE, 0>(X, src, fid, row, nface, NQFS, live);
    if constexpr (TPE > 1)
      if (part == 1) oz_gather_part<KP, NQF, TPE, 1>(X, src, fid, row, nface, NQFS, live);
    if constexpr (TPE > 2) {
      if (part == 2) oz_gather_part<KP, NQF, TPE, 2>(X, src, fid, row, nface, NQFS, live);
      if (part == 3) oz_gather_part<KP, NQF, TPE, 3>(X, src, fid, row, nface, NQFS, live);
    }
  } else {
    const int kbeg = part * KH;
    int f = kbeg / Nqf, g = kbeg - f * Nqf;
#pragma unroll
    for (int q = 0; q < KH; ++q) {
      int64_t b = 0;
      if (live && kbeg + q < NQFS) {
        b = __double_as_longlong(src[(int64_t)g * nface + fid[f * kOzM + row]]);
        if (++g == Nqf) {
          g = 0;
          ++f;
        }
      }
      X[q] = b;
    }
  }
}

// The step's A operand: this thread's KH entries of w = ucoef u + f at the
// element's nodes (raw FP64 bits); the reads are coalesced across elements.
template <int KP, int TPE>
__device__ __forceinline__ void oz_load_w(int64_t* X, const OzParams& p, int part, int64_t e,
                                          bool live) {
  constexpr int KH = KP / TPE;
#pragma unroll
  for (int q = 0; q < KH; ++q) {
    const int k = part * KH + q;
    double w = 0.0;
    if (live && k < p.n_in) {
      const int64_t i = (int64_t)k * p.nel + e;
      w = p.u[i] * p.ucoef;
      if (p.have_force) w += p.force_avg ? 0.5 * (p.force[i] + p.force_old[i]) : p.force[i];
    }
    X[q] = __double_as_longlong(w);
  }
}

// KP: K padded to 16; NQF: face points per face (0 = runtime); TPE: threads
// per element (2 or 4), each with KP / TPE entries of K and Np / TPE rows.
// MODE: kOzSweep (one eHDG iteration), kOzFinal (u = G + H uhat) or kOzStep
// (G = P w).
template <int KP, int NQF, int TPE, int MODE>
__global__ void __launch_bounds__(kOzM * TPE, 1) k_ozaki(const OzParams p) {
  constexpr int NT = kOzM * TPE;
  constexpr int KH = KP / TPE;                       // face points per thread
  constexpr int NFID = (6 + TPE - 1) / TPE;          // faces per thread (at most 6 faces)
  constexpr uint32_t SBO = 16u * KP;                 // bytes between 8-row groups
  constexpr uint32_t ABYTES = (uint32_t)kOzM * KP * 2u;
  static_assert(KH % 8 == 0, "16-byte digit chunks per thread");
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bars[5];          // empty[2], full[2], drain
  __shared__ uint32_t tmem_base;
  __shared__ int emax_sh[NT];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kOzM - 1), part = tid >> 7;
  const uint32_t bbytes = (uint32_t)p.LS * KP * 2u;                // one B slice
  unsigned char* Bs = sm;                                          // [7 * LS x KP]
  unsigned char* As = sm + kOzDigits * bbytes;                     // [2][128 x KP]
  int* fidb = reinterpret_cast<int*>(As + 2 * ABYTES);             // [2][F][128] face ids
  int* row_fg = fidb + 2 * p.F * kOzM;                             // [Np] face << 16 | point
  int* row_pt = row_fg + p.Np;                                     // [Np] element face point
  int* row_sc = row_pt + p.Np;                                     // [Np] Fb - 1074
  double* row_w = reinterpret_cast<double*>(row_sc + p.Np + (p.Np & 1));   // [Np] residual weight

  {
    const uint4* src = p.Bimg;
    uint4* dstB = reinterpret_cast<uint4*>(Bs);
    const int n16 = (int)(kOzDigits * bbytes / 16u);
    for (int i = tid; i < n16; i += NT) dstB[i] = src[i];
  }
  for (int j = tid; j < p.Np; j += NT) {
    row_sc[j] = p.Fb[j] - 1074;
    if (MODE == kOzSweep || MODE == kOzElem) {
      const int r = j < p.n_rows ? p.rows[j] : 0;
      const int f = r / p.Nqf, g = r - f * p.Nqf;
      row_fg[j] = (f << 16) | g;
      row_pt[j] = r;
      // one face Jacobian per local face: the mesh is uniform
      row_w[j] = p.face_jf[p.elem_face[(int64_t)f * p.nel]] * p.fw[g];
    }
  }
  if (tid == 0) {
    for (int b = 0; b < 5; ++b) {
      const uint32_t cnt = (b == 2 || b == 3) ? (uint32_t)NT : 1u;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[b])), "r"(cnt));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(p.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const int64_t ne = p.nel, nface = p.nface;
  // face ids of the first tile, and of this thread's faces (f = part,
  // part + TPE, ...) of the second, kept in registers
  int nfid[NFID];
  {
    const int64_t e0 = (int64_t)blockIdx.x * kOzM + row;
    const int64_t e1 = e0 + (int64_t)gridDim.x * kOzM;
#pragma unroll
    for (int m = 0; m < NFID; ++m) {
      nfid[m] = 0;
      const int f = part + TPE * m;
      if (MODE != kOzStep && f < p.F) {
        if (e0 < ne) fidb[f * kOzM + row] = p.elem_face[(int64_t)f * ne + e0];
        if (e1 < ne) nfid[m] = p.elem_face[(int64_t)f * ne + e1];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  OzCta t;
  t.As = As;
  t.empty = &bars[0];
  t.full = &bars[2];
  t.tbase = tmem_base;
  t.ph_empty[0] = t.ph_empty[1] = t.ph_full[0] = t.ph_full[1] = 0;
  t.ok = true;
  t.adesc[0] = umma_desc(smem_u32(As), 128u, SBO);
  t.adesc[1] = umma_desc(smem_u32(As + ABYTES), 128u, SBO);
  t.bdesc = umma_desc(smem_u32(Bs), 128u, SBO);
  t.bslice = bbytes >> 4;
  t.idesc_n0 = umma_idesc(1u, kOzM, 0);

  const int kk = p.it->k;                                 // read before the last block advances it
  const int64_t tlen = (int64_t)p.Nqf * nface;
  // the sweep reads uhat^k and writes uhat^{k+1}; the reconstruction uses the
  // trace of the last sweep, uhat^{k-1} after k sweeps
  const double* src = p.uhat + (int64_t)((MODE == kOzFinal ? kk + 1 : kk) & 1) * tlen;
  double* dst = p.uhat + (int64_t)((kk + 1) & 1) * tlen;
  const int64_t ntiles = (ne + kOzM - 1) / kOzM;
  const uint32_t rowoff = (uint32_t)(row >> 3) * SBO + (uint32_t)(row & 7) * 16u;
  const uint32_t kc0 = (uint32_t)(part * KH) / 8u;        // this thread's first 16-byte chunk
  const int nh = p.Np / TPE, nb = part * nh;             // this thread's rows in the epilogue
  double acc_res = 0.0;
  bool failed = false;

  int64_t X[KH];                                          // this thread's part of A's row
  {
    const int64_t e0 = (int64_t)blockIdx.x * kOzM + row;
    if (MODE == kOzStep)
      oz_load_w<KP, TPE>(X, p, part, e0, e0 < ne);
    else
      oz_gather<KP, NQF, TPE>(X, src, fidb, row, part, nface, p.NQFS, p.Nqf, e0 < ne);
  }

  int buf = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const int64_t e = tile * kOzM + row;
    const bool live = e < ne;
    int* fid = fidb + buf * p.F * kOzM;
    int* fidn = fidb + (buf ^ 1) * p.F * kOzM;
    int emax = 0;
#pragma unroll
    for (int q = 0; q < KH; ++q) emax = max(emax, (int)(((uint64_t)X[q] >> 52) & 0x7FF));
    emax_sh[tid] = emax;
    __syncthreads();
    int E = emax_sh[row];
#pragma unroll
    for (int m = 1; m < TPE; ++m) E = max(E, emax_sh[row + m * kOzM]);
    const bool bad = E == 0x7FF;                          // inf or nan among the traces
#pragma unroll
    for (int q = 0; q < KH; ++q) X[q] = oz_fixed((uint64_t)X[q], E);

    // the digit slices and their MMAs
    oz_slice<KP, TPE, 0>(t, X, rowoff, kc0, p.LS, tid);
    oz_slice<KP, TPE, 1>(t, X, rowoff, kc0, p.LS, tid);
    oz_slice<KP, TPE, 2>(t, X, rowoff, kc0, p.LS, tid);
    oz_slice<KP, TPE, 3>(t, X, rowoff, kc0, p.LS, tid);
    oz_slice<KP, TPE, 4>(t, X, rowoff, kc0, p.LS, tid);
    oz_slice<KP, TPE, 5>(t, X, rowoff, kc0, p.LS, tid);
    oz_slice<KP, TPE, 6>(t, X, rowoff, kc0, p.LS, tid);
    // the next tile's face ids (its faces of this thread from registers),
    // visible after the barrier below; prefetch the ones after
    const int64_t en = e + (int64_t)gridDim.x * kOzM;
    const int64_t enn = en + (int64_t)gridDim.x * kOzM;
#pragma unroll
    for (int m = 0; m < NFID; ++m) {
      const int f = part + TPE * m;
      if (MODE != kOzStep && f < p.F) {
        fidn[f * kOzM + row] = nfid[m];
        if (enn < ne) nfid[m] = p.elem_face[(int64_t)f * ne + enn];
      }
    }
    // slices 5 and 6: every MMA of the tile
    t.ok = mbar_wait_bounded(&t.empty[1], t.ph_empty[1], kOzWait) && t.ok;
    t.ph_empty[1] ^= 1u;
    t.ok = mbar_wait_bounded(&t.empty[0], t.ph_empty[0], kOzWait) && t.ok;
    t.ph_empty[0] ^= 1u;
    if (__syncthreads_or(t.ok ? 0 : 1)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    // the next tile's A entries are in flight during this epilogue
    if (MODE == kOzStep)
      oz_load_w<KP, TPE>(X, p, part, en, en < ne);
    else
      oz_gather<KP, NQF, TPE>(X, src, fidn, row, part, nface, p.NQFS, p.Nqf, en < ne);

    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (its elements) and
    // this thread's rows, 2 at a time (few registers while the next tile's
    // traces are in flight), all levels; the rows' Gy loads are in flight
    // during the TMEM reads
    {
      const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
      for (int n0 = nb; n0 < nb + nh; n0 += 2) {
        double gy[2], od[2];
        int64_t tix[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int n = n0 + q;
          const bool valid = live && n < p.n_rows;
          if (MODE == kOzSweep) {
            gy[q] = valid ? p.Gy[(int64_t)n * ne + e] : 0.0;
            const int fg = row_fg[n];
            tix[q] = (int64_t)(fg & 0xFFFF) * nface + fid[(fg >> 16) * kOzM + row];
            od[q] = (live && n < p.n_up) ? src[tix[q]] : 0.0;
          } else if (MODE == kOzElem) {
            gy[q] = valid ? p.Gy[(int64_t)n * ne + e] : 0.0;
          } else if (MODE == kOzFinal) {
            gy[q] = valid ? p.G[(int64_t)n * ne + e] : 0.0;
            od[q] = (valid && p.cn) ? p.u[(int64_t)n * ne + e] : 0.0;
          }
        }
        uint32_t v[kOzLevels][2];
#pragma unroll
        for (int L = 0; L < kOzLevels; ++L)
          tmem_ld2(t.tbase + lanes + (uint32_t)(L * p.LS + n0), v[L]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (live) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int n = n0 + q;
            if (n >= p.n_rows) continue;
            int64_t D[kOzLevels];
#pragma unroll
            for (int L = 0; L < kOzLevels; ++L) D[L] = __float2int_rn(__uint_as_float(v[L][q]));
            // sum_L D_L 2^(7 (6 - L)) = 2^3 (hi 2^25 + lo 2^-10), hi and lo exact
            const int64_t hi = D[0] * (1ll << 14) + D[1] * (1ll << 7) + D[2];
            const int64_t lo = D[3] * (1ll << 28) + D[4] * (1ll << 21) + D[5] * (1ll << 14) +
                               D[6] * (1ll << 7) + D[7];
            const int64_t T = hi * (1ll << 25) + (lo >> 10);
            double y = oz_to_double(T, E + row_sc[n]);
            if (bad) y = __longlong_as_double(0x7FF8000000000000ll);
            if (MODE == kOzStep) {
              p.Gout[(int64_t)n * ne + e] = y;
              continue;
            }
            if (MODE == kOzFinal) {
              const double v = gy[q] + y;
              p.u[(int64_t)n * ne + e] = p.cn ? 2.0 * v - od[q] : v;
              continue;
            }
            const double vnew = gy[q] + y;
            if (MODE == kOzSweep && n < p.n_up) {
              const int64_t ti = tix[q];
              const double dd = vnew - od[q];
              dst[ti] = vnew;
              acc_res = fma(row_w[n] * dd, dd, acc_res);
              if (p.R_out) p.R_out[ti] = (float)dd;
            } else {
              p.Y[(int64_t)row_pt[n] * ne + e] = vnew;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (failed && tid == 0) {
    atomicExch(p.err, 1);
    // drain: a commit tracks every MMA issued before it
    oz_commit(&bars[4]);
    mbar_wait_bounded(&bars[4], 0u, kOzWait);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tbase),
                 "r"(p.ncols));
  if (MODE != kOzSweep) return;
  if (p.final_here) {
    finish_residual(acc_res, p.partials, blockIdx.x, gridDim.x, p.it, p.hist, p.max_iter, p.tol,
                    p.res_scale, p.graph_mode, p.handle, gridDim.x);
  } else {
    // partial sums only; the tangential-point kernel reduces them with its own
    acc_res = fsum_warp(acc_res);
    __shared__ double red2[NT / 32];
    if ((tid & 31) == 0) red2[tid >> 5] = acc_res;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red2[w];
      p.partials[blockIdx.x] = s;
    }
  }
}

int pad16(int v) { return std::max(16, (v + 15) / 16 * 16); }

// Shape of one operator's product: `rows` output rows, K entries of A.
Ctx::OzOp oz_shape(int rows, int K) {
  Ctx::OzOp op;
  op.rows = rows;
  op.KP = pad16(K);
  op.Np = pad16(rows);
  op.LS = (op.Np + 31) / 32 * 32;
  op.ncols = 32;
  while (op.ncols < kOzLevels * op.LS) op.ncols *= 2;
  op.tpe = op.KP >= 64 ? 4 : 2;
  return op;
}

bool oz_shape_ok(const Ctx::OzOp& op, int mode) {
  const bool kp = mode == kOzStep   ? (op.KP == 16 || op.KP == 32 || op.KP == 48 || op.KP == 64)
                  : mode == kOzElem ? (op.KP == 16 || op.KP == 32)
                                    : (op.KP == 16 || op.KP == 32 || op.KP == 64 || op.KP == 96);
  return op.rows >= 1 && kp && kOzLevels * op.LS <= 512;
}

size_t oz_smem(const Ctx& c, const Ctx::OzOp& op) {
  return (size_t)kOzDigits * op.LS * op.KP * 2 + 2 * (size_t)kOzM * op.KP * 2 +
         2 * sizeof(int) * c.F * kOzM + (size_t)(3 * op.Np + (op.Np & 1)) * sizeof(int) +
         (size_t)op.Np * sizeof(double);
}

// The kernel of an operator's shape: (KP, NQF, TPE, MODE).
template <int MODE, class Fn>
cudaError_t oz_dispatch(const Ctx& c, const Ctx::OzOp& op, Fn&& fn) {
  if constexpr (MODE == kOzElem) {          // shallow water: quadrilaterals, NQFS <= 24
    return op.KP == 16 ? fn(k_ozaki<16, 0, 2, MODE>) : fn(k_ozaki<32, 0, 2, MODE>);
  } else if constexpr (MODE == kOzStep) {
    switch (op.KP) {
      case 16: return fn(k_ozaki<16, 0, 2, MODE>);
      case 32: return fn(k_ozaki<32, 0, 2, MODE>);
      case 48: return fn(k_ozaki<48, 0, 2, MODE>);
      default: return fn(k_ozaki<64, 0, 4, MODE>);
    }
  } else {
    switch (op.KP) {
      case 16: return fn(k_ozaki<16, 0, 2, MODE>);
      case 32: return fn(k_ozaki<32, 0, 2, MODE>);
      case 64:
        return c.Nqf == 9 ? fn(k_ozaki<64, 9, 4, MODE>) : fn(k_ozaki<64, 0, 4, MODE>);
      default:
        return c.Nqf == 16 ? fn(k_ozaki<96, 16, 4, MODE>) : fn(k_ozaki<96, 0, 4, MODE>);
    }
  }
}

// Digit image of the operator's rows (M with leading dimension ld; rows
// listed, or the first op.rows), and the launch shape.
template <int MODE>
cudaError_t oz_build(Ctx& c, Ctx::OzOp& op, const double* M, int ld, const int* rows, int K) {
  cudaError_t err;
  if ((err = dalloc_raw(c, &op.img, (size_t)kOzDigits * op.LS * op.KP * 2)) != cudaSuccess)
    return err;
  if ((err = dalloc_raw(c, (void**)&op.Fb, sizeof(int) * op.LS)) != cudaSuccess) return err;
  k_oz_split_rows<<<op.LS, 32, 0, c.stream>>>(M, ld, rows, op.rows, K, op.LS, op.KP,
                                               (unsigned short*)op.img, op.Fb);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  op.smem = oz_smem(c, op);
  op.threads = kOzM * op.tpe;
  // The attribute belongs to the kernel function, shared by every context
  // (and batch instance) that launches it: set it to the largest dynamic size
  // the device allows next to the kernel's static shared memory, never lower,
  // so that no context's launch is invalidated by another's smaller setting.
  int optin = 0;
  int dev = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
      cudaSuccess)
    return err;
  return oz_dispatch<MODE>(c, op, [&](auto kernel) -> cudaError_t {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if (op.smem > (size_t)dyn_max) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e != cudaSuccess) return e;
    int bpsm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, kernel, op.threads, op.smem);
    if (e != cudaSuccess) return e;
    bpsm = std::min(bpsm, 512 / op.ncols);            // TMEM columns per SM
    if (bpsm < 1) return cudaErrorInvalidConfiguration;
    const int64_t ntiles = (c.nel + kOzM - 1) / kOzM;
    op.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)bpsm * device_sms(), ntiles));
    return cudaSuccess;
  });
}

// Fields every mode reads.
OzParams oz_params(const Ctx& c, const Ctx::OzOp& op) {
  OzParams p = {};
  p.nel = c.nel;
  p.nface = c.nface;
  p.NQFS = c.NQFS;
  p.Nqf = c.Nqf;
  p.F = c.F;
  p.n_rows = op.rows;
  p.Np = op.Np;
  p.LS = op.LS;
  p.ncols = op.ncols;
  p.elem_face = c.geo.elem_face;
  p.Bimg = reinterpret_cast<const uint4*>(op.img);
  p.Fb = op.Fb;
  p.uhat = c.uhat;
  p.it = c.it;
  p.err = c.tc_err;
  return p;
}

template <int MODE>
cudaError_t oz_run(const Ctx& c, const Ctx::OzOp& op, const OzParams& p) {
  return oz_dispatch<MODE>(c, op, [&](auto kernel) -> cudaError_t {
    kernel<<<op.grid, op.threads, op.smem, c.stream>>>(p);
    return cudaGetLastError();
  });
}

}  // namespace

bool ozaki_supported(const Ctx& c) {
  if (!c.shared_op || c.F > 6) return false;
  if (c.pde == EHDG_TRANSPORT) return oz_shape_ok(oz_shape(c.n_rows, c.NQFS), kOzSweep);
  return c.pde == EHDG_SW_LINEAR && oz_shape_ok(oz_shape(c.n_rows, c.NQFS), kOzElem);
}

cudaError_t build_ozaki_operator(Ctx& c) {
  if (!ozaki_supported(c)) return cudaErrorInvalidValue;
  cudaError_t err;
  c.oz_sweep = oz_shape(c.n_rows, c.NQFS);
  err = c.pde == EHDG_TRANSPORT
            ? oz_build<kOzSweep>(c, c.oz_sweep, c.Hy, c.NQFS, c.rows, c.NQFS)
            : oz_build<kOzElem>(c, c.oz_sweep, c.Hy, c.NQFS, c.rows, c.NQFS);
  if (err != cudaSuccess) return err;
  // the reconstruction (H: n x NQFS) and the step (P: n x n), where their
  // shapes fit; otherwise they stay on the FP64 pipe
  const Ctx::OzOp fin = oz_shape(c.n, c.NQFS), stp = oz_shape(c.n, c.n);
  if (oz_shape_ok(fin, kOzFinal)) {
    c.oz_final = fin;
    if ((err = oz_build<kOzFinal>(c, c.oz_final, c.H, c.NQFS, nullptr, c.NQFS)) != cudaSuccess)
      return err;
  }
  if (oz_shape_ok(stp, kOzStep)) {
    c.oz_step = stp;
    if ((err = oz_build<kOzStep>(c, c.oz_step, c.P, c.n, nullptr, c.n)) != cudaSuccess)
      return err;
  }
  return cudaSuccess;
}

cudaError_t launch_sweep_ozaki(Ctx& c, int graph_mode, int* grid_out) {
  OzParams p = oz_params(c, c.oz_sweep);
  p.n_up = c.n_up;
  p.rows = c.rows;
  p.face_jf = c.geo.face_jf;
  fill_face_weights(c, p.fw);
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
  *grid_out = c.oz_sweep.grid;
  return oz_run<kOzSweep>(c, c.oz_sweep, p);
}

cudaError_t launch_elem_ozaki(Ctx& c) {
  OzParams p = oz_params(c, c.oz_sweep);
  p.rows = c.rows;
  p.face_jf = c.geo.face_jf;
  p.Gy = c.Gy;
  p.Y = c.Y;
  return oz_run<kOzElem>(c, c.oz_sweep, p);
}

cudaError_t launch_final_ozaki(Ctx& c) {
  OzParams p = oz_params(c, c.oz_final);
  p.G = c.G;
  p.u = c.u;
  p.cn = (c.scheme == EHDG_CN) ? 1 : 0;
  return oz_run<kOzFinal>(c, c.oz_final, p);
}

cudaError_t launch_step_ozaki(Ctx& c) {
  OzParams p = oz_params(c, c.oz_step);
  p.n_in = c.n;
  p.u = c.u;
  p.Gout = c.G;
  p.ucoef = (c.scheme == EHDG_STEADY) ? 0.0 : 1.0 / c.dt_eff;
  p.have_force = c.have_force ? 1 : 0;
  p.force_avg = (c.scheme == EHDG_CN) ? 1 : 0;
  p.force = c.force;
  p.force_old = c.force_old;
  return oz_run<kOzStep>(c, c.oz_step, p);
}

}  // namespace ehdg
