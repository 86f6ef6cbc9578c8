// Batched eHDG iteration: the iterations of many independent problems in one
// launch per kernel and iteration (Algorithm 1 of Sec. 3, run per instance).
//
// A batch's step graph runs every instance's once-per-step kernels (reset,
// right-hand side, initial trace; end-of-step reconstruction) on concurrent
// branches, and between them ONE conditional WHILE loop whose body is
//   m  correction sweeps over the tiles of every unconverged mixed-precision
//      instance (TF32/BF16 on the tensor cores, one launch each),
//   1  FP64 update uhat += delta of those instances,
//   1  FP64 sweep over the tiles of every unconverged instance,
// with the instances and their tiles in tables on the device. Each instance
// keeps its own iteration counter, residual history and stopping test: its
// residual is reduced by the last of its work items (a ticket per instance),
// exactly as its own sweep launch reduces it, and the last block of the
// launch sets the loop condition to "some instance still iterates". Converged
// instances' work items are skipped. No block waits for another.
//
// Every element's arithmetic is the single-problem path's: the FP64 sweep
// runs the same one-thread-per-element tile body (pe_tile.cuh), whose
// residual reduction is the same whatever the grid; the correction sweep
// stages the same rounded operands into the same tcgen05 MMA shapes. A
// batched instance's iterates therefore equal a solo run's bit for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ehdg_internal.h"
#include "pe_tile.cuh"
#include "step_tiles.cuh"
#include "sweep_common.cuh"
#include "tc_fx_tile.cuh"
#include "umma.cuh"

namespace ehdg {

namespace {

constexpr int kBTcM = 128;                 // elements per correction tile (MMA M)
constexpr int kBTcThreads = 256;           // two threads per element
constexpr uint32_t kBWaitLimit = 1u << 24; // mbarrier polls before giving up
constexpr int kApplyChunk = 4096;          // trace entries per update work item

struct BInst {
  // FP64 sweep (the per-element tile body of the single-problem sweep)
  int64_t nel, nface;
  int NQFS, Nqf, F, n_rows, n_up;
  int n_tiles_pe;               // 128-element tiles of the FP64 sweep
  const int* rows;
  const int32_t* elem_face;
  const double* face_jf;
  double fw[kMaxQ * kMaxQ];
  const double* Gy;
  double* Y;
  float* R_out;
  const double* Hy;
  double* uhat;
  IterState* it;
  double* partials;
  double* hist;
  double tol, res_scale;
  int max_iter;
  // corrections, mixed precision only: tensor cores (mma) or FP32 on the
  // CUDA cores, one thread per element
  int tc, mma, bf16, m;
  int Np, Kp;
  uint32_t idesc;
  const float* Hy32;
  const float* R32;
  float* d32;
  float* Y32;
  int* err;
  const uint4* Bimg;            // the rounded operator rows, K-major image (Np x Kp)
  // the sweep rows of the operator in row order, for the persistent form
  // (read through L1 instead of staged per item): [n_rows][NQFS] FP64 and,
  // with FP32 corrections, [n_up][NQFS] FP32
  const double* Hyc;
  const float* Hy32c;
  const int* rowfg;             // [Np] face | point << 8 of each row
  // fixed-shape tile body (quadrilaterals, whole faces as rows): row faces,
  // the leading ones owned, and the local face of each
  int fx, nrf, nupf;
  int rfs[6];
  // convergence time of the instance in the current step (%globaltimer), and
  // the step's start and the accumulated step times
  unsigned long long* t_conv;
  unsigned long long* t_start;
  unsigned long long* t_acc;
  int n_tiles128, n_chunks;     // work items of its correction sweeps and of its update
  // once-per-step kernels: right-hand side, initial trace, reconstruction
  int n, KE, cn;
  double ucoef;
  const double* P;
  double* u;
  const int* ey_idx;
  const double* ey_val;
  double* G;
  const double* H;
  double* uhat_n;
  const double* gb;
  double* gb_old;
  const int8_t* sgn;
  const int32_t* face_elem;
  const int8_t* face_local;
  int* step_iters;
  int* step_status;
  int step_cap;
};

// Work of the next loop iteration, rebuilt on the device after every FP64
// sweep: the instances that still iterate, with the prefix sums of their
// work items (the k-th listed instance owns items pre[k] .. pre[k+1]-1), so
// a launch visits live work only. Layout in one int array of size
// kListHeader + 5 n + 3:
//   [0] instances in the sweep list, [1] in the correction list (mixed
//   precision), then act_sw[n], pre_sw[n+1], act_mx[n], pre_tc[n+1], pre_ap[n+1].
constexpr int kListHeader = 2;
struct ListView {
  int n;
  template <class T> __device__ T* act_sw(T* L) const { return L + kListHeader; }
  template <class T> __device__ T* pre_sw(T* L) const { return L + kListHeader + n; }
  template <class T> __device__ T* act_mx(T* L) const { return L + kListHeader + 2 * n + 1; }
  template <class T> __device__ T* pre_tc(T* L) const { return L + kListHeader + 3 * n + 1; }
  template <class T> __device__ T* pre_ap(T* L) const { return L + kListHeader + 4 * n + 2; }
};

// Rebuild the lists from the instances' continue flags (one block): each
// thread takes a contiguous run of instances, counts its run's work, the runs'
// offsets come from a scan over the threads, and each thread writes its run.
// counts[i] = (sweep items, 1 if mixed precision, correction tiles, update
// chunks) of instance i.
__device__ void build_lists(const BInst* inst, const int4* counts, int n_inst, int* L) {
  extern __shared__ double sm[];
  const ListView v{n_inst};
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  int* part = reinterpret_cast<int*>(sm);           // [5][nt]: per-thread sums, then offsets
  __syncthreads();
  const int per = (n_inst + nt - 1) / nt;
  const int i0 = min(n_inst, tid * per), i1 = min(n_inst, i0 + per);
  int ns = 0, nm = 0, ps = 0, pt = 0, pa = 0;
  for (int i = i0; i < i1; ++i) {
    if (!reinterpret_cast<volatile IterState*>(inst[i].it)->cont) continue;
    const int4 c = counts[i];
    ++ns;
    ps += c.x;
    if (c.y) {
      ++nm;
      pt += c.z;
      pa += c.w;
    }
  }
  part[0 * nt + tid] = ns;
  part[1 * nt + tid] = nm;
  part[2 * nt + tid] = ps;
  part[3 * nt + tid] = pt;
  part[4 * nt + tid] = pa;
  __syncthreads();
  if (tid < 5) {             // exclusive scan of each quantity over the threads
    int run = 0;
    for (int t = 0; t < nt; ++t) {
      const int x = part[tid * nt + t];
      part[tid * nt + t] = run;
      run += x;
    }
    if (tid == 0) L[0] = run;
    if (tid == 1) L[1] = run;
  }
  __syncthreads();
  const int ons = part[0 * nt + tid], onm = part[1 * nt + tid];
  int ops = part[2 * nt + tid], opt = part[3 * nt + tid], opa = part[4 * nt + tid];
  int ks = ons, km = onm;
  int* act_sw = v.act_sw(L);
  int* pre_sw = v.pre_sw(L);
  int* act_mx = v.act_mx(L);
  int* pre_tc = v.pre_tc(L);
  int* pre_ap = v.pre_ap(L);
  for (int i = i0; i < i1; ++i) {
    if (!reinterpret_cast<volatile IterState*>(inst[i].it)->cont) continue;
    const int4 c = counts[i];
    act_sw[ks] = i;
    pre_sw[ks] = ops;
    ops += c.x;
    ++ks;
    if (c.y) {
      act_mx[km] = i;
      pre_tc[km] = opt;
      pre_ap[km] = opa;
      opt += c.z;
      opa += c.w;
      ++km;
    }
  }
  if (tid == nt - 1) {       // the totals close the prefix arrays
    pre_sw[ks] = ops;
    pre_tc[km] = opt;
    pre_ap[km] = opa;
  }
  __threadfence();
  __syncthreads();
}

// Which listed instance owns item w: the last k with pre[k] <= w (binary
// search over the prefix sums, k < count).
__device__ __forceinline__ int owner_of(const int* pre, int count, int w) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One FP64 sweep of every instance that still iterates: items = (instance,
// 128-element tile) from the lists; the instance's own single-problem tile
// body, reduction and stopping test.
__global__ void __launch_bounds__(kPeTile) k_batch_sweep(const BInst* inst, const int4* counts,
                                                          int* lists, int n_inst,
                                                          unsigned int* ticket, int graph_mode,
                                                          cudaGraphConditionalHandle handle) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x;
  const ListView lv{n_inst};
  const int n_act = lists[0];
  const int* act = lv.act_sw(lists);
  const int* pre = lv.pre_sw(lists);
  const int n_items = n_act > 0 ? pre[n_act] : 0;
  int cur = -1;
  double* Hsh = sm;                                   // the instance's sweep rows [n_rows][NQ]
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    // every listed instance iterates; its state cannot change before all its
    // work items are done
    const int k = owner_of(pre, n_act, w);
    const int idx = act[k];
    const int64_t tile = w - pre[k];
    const BInst& I = inst[idx];
    const int nq = I.NQFS;
    if (idx != cur) {   // the previous item's threads are past its last barrier
      for (int i = tid; i < I.n_rows * nq; i += kPeTile) {
        const int j = i / nq, c = i - j * nq;
        Hsh[i] = I.Hy[I.rows[j] * nq + c];
      }
      __syncthreads();
      cur = idx;
    }
    const int kk = reinterpret_cast<volatile IterState*>(I.it)->k;
    const int64_t tlen = (int64_t)I.Nqf * I.nface;
    PeView v = {};
    v.nel = I.nel;
    v.nface = I.nface;
    v.n_rows = I.n_rows;
    v.n_up = I.n_up;
    v.rows = I.rows;
    v.elem_face = I.elem_face;
    v.face_jf = I.face_jf;
    v.fw = I.fw;
    v.Gy = I.Gy;
    v.Y = I.Y;
    v.R_out = I.R_out;
    v.partials = I.partials;
    v.it = I.it;
    v.hist = I.hist;
    v.max_iter = I.max_iter;
    v.tol = I.tol;
    v.res_scale = I.res_scale;
    v.uhat = I.uhat;
    const double* src = I.uhat + (int64_t)(kk & 1) * tlen;
    double* dst = I.uhat + (int64_t)((kk + 1) & 1) * tlen;
    const int64_t ntiles = I.n_tiles_pe;
    bool last;
    switch (nq) {
      case 8: last = pe_tile<8>(v, Hsh, src, dst, tile, ntiles, 0, handle); break;
      case 12: last = pe_tile<12>(v, Hsh, src, dst, tile, ntiles, 0, handle); break;
      case 16: last = pe_tile<16>(v, Hsh, src, dst, tile, ntiles, 0, handle); break;
      case 20: last = pe_tile<20>(v, Hsh, src, dst, tile, ntiles, 0, handle); break;
      case 24: last = pe_tile<24>(v, Hsh, src, dst, tile, ntiles, 0, handle); break;
      default: last = pe_tile<28>(v, Hsh, src, dst, tile, ntiles, 0, handle); break;
    }
    if (last && tid == 0 && !reinterpret_cast<volatile IterState*>(I.it)->cont)
      *I.t_conv = global_ns();
  }
  // the last block of the launch: is any instance still iterating?
  __shared__ bool s_last;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the next iteration's work, and the loop condition
  build_lists(inst, counts, n_inst, lists);
  if (tid == 0) {
    *ticket = 0u;
    if (graph_mode) cudaGraphSetConditional(handle, lists[0] > 0 ? 1u : 0u);
  }
}

// The work lists at the start of a step's loop (after the instances' reset,
// right-hand side and, for mixed precision, first FP64 sweep).
__global__ void k_batch_lists(const BInst* inst, const int4* counts, int n_inst, int* lists) {
  build_lists(inst, counts, n_inst, lists);
}

__device__ __forceinline__ uint32_t b_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// 16 bytes of one K-major core-matrix row: 4 TF32 or 8 BF16 values
__device__ __forceinline__ void b_store_chunk(unsigned char* dst, const float* v, int bf16) {
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
        make_uint4(b_to_tf32(v[0]), b_to_tf32(v[1]), b_to_tf32(v[2]), b_to_tf32(v[3]));
  }
}

__device__ __forceinline__ void b_store_elem(unsigned char* base, int row, int k, int esize,
                                             uint32_t sbo, float v, int bf16) {
  const uint32_t off = kmajor_off(row, k * esize, sbo);
  if (bf16) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
  } else {
    *reinterpret_cast<uint32_t*>(base + off) = b_to_tf32(v);
  }
}

// One 128-element tile of instance I's correction sweep j in the fixed-shape
// tile body of the single-problem sweep (quadrilaterals, NQF points per face,
// two threads per element; part Q = the thread's half of the tile).
template <int NQF, int BF16, int Q>
__device__ __forceinline__ void btc_fx_part(const BInst& I, int j, unsigned char* As,
                                            unsigned char* Bs, uint64_t* mbar, uint32_t tbase,
                                            uint32_t& phase, bool& failed, int64_t tile) {
  TcFxParams q;
  q.nel = I.nel;
  q.nface = (uint32_t)I.nface;
  q.n_rf = I.nrf;
  q.n_up_f = I.nupf;
#pragma unroll
  for (int i = 0; i < 6; ++i) q.rfs[i] = I.rfs[i];
  q.Np = I.Np;
  q.ncols = 0;
  q.idesc = I.idesc;
  q.elem_face = I.elem_face;
  q.img = I.Bimg;
  const int64_t trace = (int64_t)I.Nqf * I.nface;
  q.R = I.R32;
  q.in = j == 0 ? I.R32 : I.d32 + (int64_t)((j - 1) & 1) * trace;
  q.out = I.d32 + (int64_t)(j & 1) * trace;
  q.Y32 = I.Y32;
  q.err = I.err;
  q.apply_uhat = nullptr;     // the batched loop's FP64 update is its own launch
  q.apply_k = nullptr;
  q.apply_total = 0;
  const int64_t e = tile * kFxM + (threadIdx.x & (kFxM - 1));
  int fid[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) fid[f] = e < I.nel ? I.elem_face[f * I.nel + e] : 0;
  fx_tile<4, NQF, BF16, 2, Q>(q, As, Bs, mbar, tbase, phase, failed, tile, fid);
}

template <int NQF, int BF16>
__device__ __forceinline__ void btc_fx(const BInst& I, int j, unsigned char* As,
                                       unsigned char* Bs, uint64_t* mbar, uint32_t tbase,
                                       uint32_t& phase, bool& failed, int64_t tile) {
  // the halves are warp-uniform (128 threads each)
  if ((threadIdx.x >> 7) == 0)
    btc_fx_part<NQF, BF16, 0>(I, j, As, Bs, mbar, tbase, phase, failed, tile);
  else
    btc_fx_part<NQF, BF16, 1>(I, j, As, Bs, mbar, tbase, phase, failed, tile);
}

// Inner correction sweep j of every unconverged TF32/BF16 mixed-precision
// instance: delta_out = R + (delta_in Hy^T at the rows), owner writes; items[w]
// = (instance, 128-element tile). The operands, MMA shapes and epilogue are
// those of the single-problem tensor-core correction sweep.
__global__ void __launch_bounds__(kBTcThreads) k_batch_tc(const BInst* inst, const int* lists,
                                                          int n_inst, int j, int ncols,
                                                          int smem_b, int smem_a) {
  extern __shared__ __align__(1024) unsigned char smb[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kBTcM - 1), half = tid >> 7;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;
  unsigned char* Bs = smb;                          // Np x Kp of the current instance
  unsigned char* As = smb + smem_b;                 // 128 x Kp
  int* fid = reinterpret_cast<int*>(As + smem_a);   // [F][128]
  int* row_f = fid + 6 * kBTcM;                     // [Np] face of a row
  int* row_g = row_f + 256;                         // [Np] point of a row
  uint32_t phase = 0;
  bool failed = false;
  int cur = -1;
  const ListView lv{n_inst};
  const int n_act = lists[1];
  const int* act = lv.act_mx(lists);
  const int* pre = lv.pre_tc(lists);
  const int n_items = n_act > 0 ? pre[n_act] : 0;
  // a contiguous run of items per block: consecutive tiles of one instance
  // share its staged operator
  const int per = (n_items + gridDim.x - 1) / gridDim.x;
  const int w_end = min(n_items, (int)(blockIdx.x + 1) * per);
  for (int w = blockIdx.x * per; w < w_end && !failed; ++w) {
    const int k = owner_of(pre, n_act, w);
    const int2 item = make_int2(act[k], w - pre[k]);
    const BInst& I = inst[item.x];
    if (!I.mma || I.m <= j) continue;               // FP32 corrections, or its inner sweeps done
    __syncthreads();   // the previous item is done with the shared operands
    const int esize = I.bf16 ? 2 : 4;
    const uint32_t kbytes = (uint32_t)I.Kp * esize;
    const uint32_t sbo = kbytes * 8u;
    if (item.x != cur) {
      // the instance's operator rows (B, rounded once at setup) and row tables
      for (int jj = tid; jj < I.Np; jj += kBTcThreads) {
        const int fg = I.rowfg[jj];
        row_f[jj] = fg & 255;
        row_g[jj] = fg >> 8;
      }
      const int n16 = (int)((uint32_t)I.Np * kbytes / 16u);
      for (int i = tid; i < n16; i += kBTcThreads)
        reinterpret_cast<uint4*>(Bs)[i] = I.Bimg[i];
      cur = item.x;
    }
    if (I.fx) {
      // the fixed-shape tile body (the single-problem sweep's, bit for bit)
#define EHDG_BTC_FX(N)                                                                   \
  case N:                                                                                \
    if (I.bf16)                                                                          \
      btc_fx<N, 1>(I, j, As, Bs, &mbar, tbase, phase, failed, item.y);                   \
    else                                                                                 \
      btc_fx<N, 0>(I, j, As, Bs, &mbar, tbase, phase, failed, item.y);                   \
    break;
      switch (I.Nqf) {
        EHDG_BTC_FX(2)
        EHDG_BTC_FX(3)
        EHDG_BTC_FX(4)
        EHDG_BTC_FX(5)
        EHDG_BTC_FX(6)
        EHDG_BTC_FX(7)
        default: break;
      }
#undef EHDG_BTC_FX
      asm volatile("tcgen05.fence::before_thread_sync;");
      continue;
    }
    const int64_t trace = (int64_t)I.Nqf * I.nface;
    const float* in = j == 0 ? I.R32 : I.d32 + (int64_t)((j - 1) & 1) * trace;
    float* out = I.d32 + (int64_t)(j & 1) * trace;
    const int64_t ne = I.nel, nface = I.nface;
    const int64_t e = (int64_t)item.y * kBTcM + row;
    __syncthreads();
    if (e < ne)
      for (int f = half; f < I.F; f += 2) fid[f * kBTcM + row] = I.elem_face[f * ne + e];
    __syncthreads();
    {
      // A: this tile's correction values at its elements' face points, each
      // element's K range split between its two threads
      const uint32_t rowoff = (uint32_t)(row >> 3) * sbo + (uint32_t)(row & 7) * 16u;
      const int khalf = I.Kp / 2;
      const int kbeg = half * khalf, kend = kbeg + khalf;
      int f = kbeg / I.Nqf, g = kbeg - (kbeg / I.Nqf) * I.Nqf;
      for (int k0 = kbeg; k0 < kend; k0 += 16) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float x = 0.f;
          if (e < ne && k0 + q < I.NQFS && k0 + q < kend) {
            x = in[g * nface + fid[f * kBTcM + row]];
            if (++g == I.Nqf) {
              g = 0;
              ++f;
            }
          }
          v[q] = x;
        }
        if (I.bf16) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (k0 + 8 * h < kend)
              b_store_chunk(As + rowoff + (uint32_t)((k0 + 8 * h) / 8) * 128u, v + 8 * h, 1);
        } else {
#pragma unroll
          for (int h = 0; h < 4; ++h)
            if (k0 + 4 * h < kend)
              b_store_chunk(As + rowoff + (uint32_t)((k0 + 4 * h) / 4) * 128u, v + 4 * h, 0);
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
        if (I.bf16) {
          asm volatile(
              "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tbase),
              "l"(ad), "l"(bd), "r"(I.idesc), "r"(acc));
        } else {
          asm volatile(
              "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}\n" ::"r"(tbase),
              "l"(ad), "l"(bd), "r"(I.idesc), "r"(acc));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar)));
    }
    uint32_t ok = 1;
    if (tid == 0) ok = mbar_wait_bounded(&mbar, phase, kBWaitLimit) ? 1u : 0u;
    if (__syncthreads_or(ok ? 0 : 1)) {
      if (tid == 0) atomicExch(I.err, 1);
      failed = true;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
      const int nhalf = I.Np / 2;
      const int cbeg = half * nhalf, cend = cbeg + nhalf;
      for (int c0 = cbeg; c0 < cend; c0 += 8) {
        uint32_t v[8];
        tmem_ld8(tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (e < ne) {
          int64_t pt[8];
          float rv[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int jr = c0 + q;
            pt[q] = -1;
            rv[q] = 0.f;
            if (jr < I.n_rows && jr < I.n_up) {
              pt[q] = (int64_t)row_g[jr] * nface + fid[row_f[jr] * kBTcM + row];
              rv[q] = I.R32[pt[q]];
            }
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int jr = c0 + q;
            if (jr >= I.n_rows) break;
            const float acc = __uint_as_float(v[q]);
            if (pt[q] >= 0) {
              out[pt[q]] = rv[q] + acc;
            } else {
              I.Y32[(int64_t)(row_f[jr] * I.Nqf + row_g[jr]) * ne + e] = acc;
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
                 "r"(ncols));
}

// Setup of the persistent form: instance i's sweep rows in row order
__global__ void k_batch_rows(const double* Hy, const float* Hy32, const int* rows, int n_rows,
                             int n_up, int NQFS, double* Hyc, float* Hy32c) {
  for (int t = threadIdx.x; t < n_rows * NQFS; t += blockDim.x) {
    const int j = t / NQFS, c = t - j * NQFS;
    Hyc[t] = Hy[rows[j] * NQFS + c];
    if (Hy32c && j < n_up) Hy32c[t] = Hy32[rows[j] * NQFS + c];
  }
}

// Setup: instance i's operator rows rounded to TF32 / BF16 in the K-major
// image the correction sweep stages (the single-problem sweep's rounding),
// and its row tables.
__global__ void k_batch_bimg(const float* Hy32, const int* rows, int n_rows, int NQFS, int Nqf,
                             int Np, int Kp, int bf16, unsigned char* img, int* rowfg) {
  const int esize = bf16 ? 2 : 4;
  const uint32_t sbo = (uint32_t)Kp * esize * 8u;
  for (int i = threadIdx.x; i < Np * Kp; i += blockDim.x) {
    const int n = i / Kp, k = i - n * Kp;
    float v = 0.f;
    if (n < n_rows && k < NQFS) v = Hy32[rows[n] * NQFS + k];
    b_store_elem(img, n, k, esize, sbo, v, bf16);
  }
  for (int jj = threadIdx.x; jj < Np; jj += blockDim.x) {
    const int r = jj < n_rows ? rows[jj] : 0;
    rowfg[jj] = (r / Nqf) | ((r - (r / Nqf) * Nqf) << 8);
  }
}

// Inner correction sweep j of every instance that still iterates with FP32
// corrections (the single-problem one-thread-per-element tile body); items
// from the same list as the tensor-core sweep (128-element tiles).
__global__ void __launch_bounds__(kPeTile) k_batch_lp(const BInst* inst, const int* lists,
                                                      int n_inst, int j) {
  extern __shared__ float smf[];
  const ListView lv{n_inst};
  const int n_act = lists[1];
  const int* act = lv.act_mx(lists);
  const int* pre = lv.pre_tc(lists);
  const int n_items = n_act > 0 ? pre[n_act] : 0;
  int cur = -1;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int k = owner_of(pre, n_act, w);
    const int idx = act[k];
    const BInst& I = inst[idx];
    if (I.mma || I.m <= j) continue;
    const int nq = I.NQFS;
    if (idx != cur) {
      __syncthreads();
      for (int i = threadIdx.x; i < I.n_up * nq; i += kPeTile) {
        const int jj = i / nq, c = i - jj * nq;
        smf[i] = I.Hy32[I.rows[jj] * nq + c];
      }
      __syncthreads();
      cur = idx;
    }
    const int64_t trace = (int64_t)I.Nqf * I.nface;
    LpPeView v;
    v.nel = I.nel;
    v.nface = I.nface;
    v.n_up = I.n_up;
    v.rows = I.rows;
    v.elem_face = I.elem_face;
    v.R = I.R32;
    v.in = j == 0 ? I.R32 : I.d32 + (int64_t)((j - 1) & 1) * trace;
    v.out = I.d32 + (int64_t)(j & 1) * trace;
    const int64_t tile = w - pre[k];
    switch (nq) {
      case 8: lp_pe_tile<8>(v, smf, tile); break;
      case 12: lp_pe_tile<12>(v, smf, tile); break;
      case 16: lp_pe_tile<16>(v, smf, tile); break;
      case 20: lp_pe_tile<20>(v, smf, tile); break;
      case 24: lp_pe_tile<24>(v, smf, tile); break;
      default: lp_pe_tile<28>(v, smf, tile); break;
    }
  }
}

// uhat <- uhat + delta in FP64 for every unconverged mixed-precision
// instance (the single-problem update, slot k&1 = slot (k+1)&1 + delta of
// its last inner sweep); items[w] = (instance, chunk of kApplyChunk entries).
__global__ void __launch_bounds__(256) k_batch_apply(const BInst* inst, const int* lists,
                                                     int n_inst) {
  const ListView lv{n_inst};
  const int n_act = lists[1];
  const int* act = lv.act_mx(lists);
  const int* pre = lv.pre_ap(lists);
  const int n_items = n_act > 0 ? pre[n_act] : 0;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int k = owner_of(pre, n_act, w);
    const int2 item = make_int2(act[k], w - pre[k]);
    const BInst& I = inst[item.x];
    const int K = reinterpret_cast<volatile IterState*>(I.it)->k;
    const int64_t total = (int64_t)I.Nqf * I.nface;
    double* dst = I.uhat + (int64_t)(K & 1) * total;
    const double* src = I.uhat + (int64_t)((K + 1) & 1) * total;
    const float* delta = I.d32 + (int64_t)((I.m - 1) & 1) * total;
    const int64_t t0 = (int64_t)item.y * kApplyChunk;
    const int64_t t1 = std::min<int64_t>(t0 + kApplyChunk, total);
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) dst[t] = src[t] + (double)delta[t];
  }
}

// ---------------------------------------------------------------------------
// Persistent form (FP64 and FP32-correction instances): every iteration of a
// step in ONE launch. Each instance moves through its own stages -- the FP64
// sweep, then for mixed precision its m correction sweeps and the FP64 update,
// then the next FP64 sweep -- at its own pace: the block that completes an
// instance's stage publishes the next stage's work items into a ring in device
// memory, and every block takes the next item of the ring, whatever its
// instance. A stage's items are published only after every item of the
// instance's previous stage is done, and they run the same tile bodies as the
// loop, so every instance computes its solo run's iterates bit for bit. No
// block waits for another block's progress except through the ring, whose
// polls are bounded: a wait that gives up sets an error flag and its block
// leaves (the step then reports EHDG_ERR_TIMEOUT).
// ---------------------------------------------------------------------------
constexpr int kQCap = 1 << 16;                  // ring slots (a power of two)
constexpr unsigned int kQWaitLimit = 1u << 24;  // polls of one slot before giving up
// stage codes (an item packs stage << 24 | index, positive): 0 the FP64 sweep,
// 1..m correction sweep s - 1 (m <= 64), 127 the FP64 update
constexpr int kStSweep = 0, kStApply = 127;

struct BQueue {
  unsigned long long head;      // items claimed (monotonic over the batch's life)
  unsigned long long tail;      // items published
  int live;                     // instances still iterating in the current step
  int err;                      // a poll gave up
};

__device__ __forceinline__ long long q_ld_acquire(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void q_st_release(long long* p, long long v) {
  asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Publish n items (inst, stage, 0..n-1): ring positions from one reservation
// on the tail, each slot's payload before its sequence number (release).
// Every thread of the block calls this.
__device__ void q_publish(BQueue* q, long long* seq, int2* items, int inst, int stage, int n) {
  __shared__ unsigned long long s_start;
  if (threadIdx.x == 0) s_start = atomicAdd(&q->tail, (unsigned long long)n);
  __syncthreads();
  const unsigned long long st = s_start;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const unsigned long long w = st + (unsigned long long)k;
    const int slot = (int)(w & (unsigned long long)(kQCap - 1));
    items[slot] = make_int2(inst, (stage << 24) | k);
    q_st_release(seq + slot, (long long)w);
  }
  __syncthreads();
}

// A correction item covers up to kQCorrTiles consecutive 128-element tiles
// (its block runs them one after the other): the FP32 tile is short, and one
// item per tile would spend more on taking and completing items than on the
// tile.
constexpr int kQCorrTiles = 4;
__device__ __forceinline__ int corr_items(const BInst& I) {
  return (I.n_tiles128 + kQCorrTiles - 1) / kQCorrTiles;
}

// the first stage of an instance that still iterates after the pre-loop sweep
__device__ __forceinline__ int2 first_stage(const BInst& I) {
  return (I.tc && !I.mma && I.m > 0) ? make_int2(1, corr_items(I)) : make_int2(kStSweep, I.n_tiles_pe);
}

// Start of a step's persistent loop (one block): claims restart at the
// published end, and every instance the pre-loop sweep left iterating gets
// its first stage.
__global__ void k_batch_qinit(const BInst* inst, int n_inst, BQueue* q, long long* seq,
                              int2* items, int* stage_cnt) {
  if (threadIdx.x == 0) {
    q->head = q->tail;
    q->live = 0;
    q->err = 0;
  }
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) stage_cnt[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const BInst& I = inst[i];
    if (!reinterpret_cast<volatile IterState*>(I.it)->cont) continue;
    atomicAdd(&q->live, 1);
    const int2 st = first_stage(I);
    const unsigned long long s0 = atomicAdd(&q->tail, (unsigned long long)st.y);
    for (int k = 0; k < st.y; ++k) {
      const unsigned long long w = s0 + (unsigned long long)k;
      const int slot = (int)(w & (unsigned long long)(kQCap - 1));
      items[slot] = make_int2(i, (st.x << 24) | k);
      q_st_release(seq + slot, (long long)w);
    }
  }
}

template <int NQ>
__device__ __forceinline__ bool q_sweep_item(const BInst& I, const double* Hsh, int64_t tile) {
  PeView v = {};
  v.nel = I.nel;
  v.nface = I.nface;
  v.n_rows = I.n_rows;
  v.n_up = I.n_up;
  v.rows = I.rows;
  v.elem_face = I.elem_face;
  v.face_jf = I.face_jf;
  v.fw = I.fw;
  v.Gy = I.Gy;
  v.Y = I.Y;
  v.R_out = I.R_out;
  v.partials = I.partials;
  v.it = I.it;
  v.hist = I.hist;
  v.max_iter = I.max_iter;
  v.tol = I.tol;
  v.res_scale = I.res_scale;
  v.uhat = I.uhat;
  const int kk = reinterpret_cast<volatile IterState*>(I.it)->k;
  const int64_t tlen = (int64_t)I.Nqf * I.nface;
  const double* src = I.uhat + (int64_t)(kk & 1) * tlen;
  double* dst = I.uhat + (int64_t)((kk + 1) & 1) * tlen;
  return pe_tile<NQ, true>(v, Hsh, src, dst, tile, I.n_tiles_pe, 0, 0);
}

template <int NQ>
__device__ __forceinline__ void q_corr_item(const BInst& I, const float* Hsh32, int j,
                                            int64_t tile) {
  const int64_t trace = (int64_t)I.Nqf * I.nface;
  LpPeView v;
  v.nel = I.nel;
  v.nface = I.nface;
  v.n_up = I.n_up;
  v.rows = I.rows;
  v.elem_face = I.elem_face;
  v.R = I.R32;
  v.in = j == 0 ? I.R32 : I.d32 + (int64_t)((j - 1) & 1) * trace;
  v.out = I.d32 + (int64_t)(j & 1) * trace;
  lp_pe_tile<NQ, true>(v, Hsh32, tile);
}

// five resident blocks per SM (96 registers; four at the unconstrained 128):
// the blocks spend much of an item at barriers while one thread takes the
// next item or counts the stage, so more blocks keep the pipes busier
__global__ void __launch_bounds__(kPeTile, 5) k_batch_persist(const BInst* inst, BQueue* q,
                                                           long long* seq, int2* items,
                                                           int* stage_cnt, unsigned int limit) {
  __shared__ int2 s_item;
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  // thread 0's claim of the next ring position; a correction or update item
  // takes it together with its stage count (two atomics in flight at once)
  unsigned long long w = 0ull;
  bool claimed = false;
  for (;;) {
    if (tid == 0) {
      if (!claimed) w = atomicAdd(&q->head, 1ull);
      claimed = false;
      const int slot = (int)(w & (unsigned long long)(kQCap - 1));
      int go = 0;
      for (unsigned int n = 0;; ++n) {
        if (q_ld_acquire(seq + slot) == (long long)w) {
          s_item = __ldcg(items + slot);   // ordered after the acquire
          go = 1;
          break;
        }
        if (*reinterpret_cast<volatile int*>(&q->live) == 0 ||
            *reinterpret_cast<volatile int*>(&q->err) != 0)
          break;
        if (n >= limit) {
          atomicExch(&q->err, 1);
          break;
        }
        if (n >= 32) __nanosleep(128);
      }
      s_flag = go;
    }
    __syncthreads();
    if (!s_flag) break;
    const int2 item = s_item;
    const int i = item.x, stage = (int)((unsigned int)item.y >> 24), idx = item.y & 0xFFFFFF;
    const BInst& I = inst[i];
    const int nq = I.NQFS;
    const int kind = stage == kStSweep ? 0 : (stage == kStApply ? 2 : 1);
    // the operator rows come through L1 (every thread of a row reads the same
    // entry), not staged per item: consecutive items are mostly of other
    // instances
    bool done;
    if (kind == 0) {
      const double* hr = I.Hyc;
      switch (nq) {
        case 8: done = q_sweep_item<8>(I, hr, idx); break;
        case 12: done = q_sweep_item<12>(I, hr, idx); break;
        case 16: done = q_sweep_item<16>(I, hr, idx); break;
        case 20: done = q_sweep_item<20>(I, hr, idx); break;
        case 24: done = q_sweep_item<24>(I, hr, idx); break;
        default: done = q_sweep_item<28>(I, hr, idx); break;
      }
    } else {
      if (kind == 1) {
        const float* smf = I.Hy32c;
        const int j = stage - 1;
        const int t1 = min((idx + 1) * kQCorrTiles, I.n_tiles128);
        for (int tile = idx * kQCorrTiles; tile < t1; ++tile) {
          switch (nq) {
            case 8: q_corr_item<8>(I, smf, j, tile); break;
            case 12: q_corr_item<12>(I, smf, j, tile); break;
            case 16: q_corr_item<16>(I, smf, j, tile); break;
            case 20: q_corr_item<20>(I, smf, j, tile); break;
            case 24: q_corr_item<24>(I, smf, j, tile); break;
            default: q_corr_item<28>(I, smf, j, tile); break;
          }
        }
      } else {
        // the FP64 update (the loop's k_batch_apply on one chunk)
        const int K = reinterpret_cast<volatile IterState*>(I.it)->k;
        const int64_t total = (int64_t)I.Nqf * I.nface;
        double* dst = I.uhat + (int64_t)(K & 1) * total;
        const double* src = I.uhat + (int64_t)((K + 1) & 1) * total;
        const float* delta = I.d32 + (int64_t)((I.m - 1) & 1) * total;
        const int64_t t0 = (int64_t)idx * kApplyChunk;
        const int64_t t1 = std::min<int64_t>(t0 + kApplyChunk, total);
        for (int64_t t = t0 + tid; t < t1; t += kPeTile)
          dst[t] = __ldcg(src + t) + (double)__ldcg(delta + t);
      }
      // the stage is done when its last item is
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        const int n = kind == 2 ? I.n_chunks : corr_items(I);
        const int c = atomicAdd(&stage_cnt[i], 1);
        w = atomicAdd(&q->head, 1ull);   // polled after any publish below
        claimed = true;
        const int last = c == n - 1;
        if (last) {
          stage_cnt[i] = 0;
          __threadfence();
        }
        s_flag = last;
      }
      __syncthreads();
      done = s_flag != 0;
    }
    if (!done) continue;
    // the instance's next stage, or its end in this step
    if (tid == 0) {
      int2 nx = make_int2(-1, 0);
      if (kind == 0) {
        if (reinterpret_cast<volatile IterState*>(I.it)->cont) {
          nx = first_stage(I);
        } else {
          *I.t_conv = global_ns();
          __threadfence();
          atomicSub(&q->live, 1);
        }
      } else if (kind == 1) {
        nx = (stage < I.m) ? make_int2(stage + 1, corr_items(I)) : make_int2(kStApply, I.n_chunks);
      } else {
        nx = make_int2(kStSweep, I.n_tiles_pe);
      }
      s_item = nx;
    }
    __syncthreads();
    const int2 nx = s_item;
    __syncthreads();
    if (nx.x >= 0) q_publish(q, seq, items, i, nx.x, nx.y);
  }
}

// ---------------------------------------------------------------------------
// Once-per-step kernels of the looped instances, each one launch for all of
// them; static work lists: pre[i] .. pre[i+1]-1 are instance i's items.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int static_owner(const int* pre, int n, int w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// iteration state reset (the single-problem reset) and the step's start time
__global__ void k_batch_begin(const BInst* inst, int n_inst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  const BInst& I = inst[i];
  IterState* it = I.it;
  it->k = 0;
  it->cont = 1;
  it->status = EHDG_OK;
  it->counter = 0u;
  it->bar = 0u;
  it->abort = 0;
  it->r_last = 0.0;
  *I.t_start = global_ns();
  *I.t_conv = 0ull;
}

__device__ StepParams step_params(const BInst& I) {
  StepParams p = {};
  p.nel = I.nel;
  p.n = I.n;
  p.NQFS = I.NQFS;
  p.KE = I.KE;
  p.shared = 1;
  p.ucoef = I.ucoef;
  p.P = I.P;
  p.u = I.u;
  p.ey_idx = I.ey_idx;
  p.ey_val = I.ey_val;
  p.rows = I.rows;
  p.n_rows = I.n_rows;
  p.G = I.G;
  p.Gy = const_cast<double*>(I.Gy);
  p.Y = I.Y;
  return p;
}

// the step's right-hand side G = P w, Gy and Y0 (items: 32-element tiles)
__global__ void __launch_bounds__(32 * kStepT) k_batch_step(const BInst* inst, const int* pre,
                                                            int n_inst, int nmax) {
  extern __shared__ double sm[];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  double* Psh = sm;                                   // [n][n]
  double* w = Psh + nmax * nmax;                      // [n][32]
  double* g = w + nmax * 32;                          // [n][32]
  const int n_items = pre[n_inst];
  int cur = -1;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int i = static_owner(pre, n_inst, it);
    const BInst& I = inst[i];
    if (i != cur) {   // step_tile starts and ends with barriers around its use of Psh
      __syncthreads();
      for (int k = tid; k < I.n * I.n; k += 32 * kStepT) Psh[k] = I.P[k];
      cur = i;
    }
    step_tile(step_params(I), Psh, w, g, nullptr, it - pre[i]);
  }
}

// the initial trace (the trace formula of u^n with the new boundary data),
// written to both trace slots (items: chunks of kApplyChunk face points)
__global__ void __launch_bounds__(256) k_batch_trace0(const BInst* inst, const int* pre,
                                                      int n_inst) {
  const int n_items = pre[n_inst];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int i = static_owner(pre, n_inst, it);
    const BInst& I = inst[i];
    const int64_t total = (int64_t)I.Nqf * I.nface;
    const int64_t t0 = (int64_t)(it - pre[i]) * kApplyChunk;
    const int64_t t1 = std::min<int64_t>(t0 + kApplyChunk, total);
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      const int gf = (int)(t / I.nface);
      const int64_t face = t - (int64_t)gf * I.nface;
      const double uh = transport_trace_point(I.nel, I.nface, I.Nqf, I.cn, I.face_elem,
                                              I.face_local, I.sgn, I.Y, I.gb, I.gb_old, gf,
                                              face);
      I.uhat[total + t] = uh;
      I.uhat[t] = uh;
    }
  }
}

// the reconstruction u^{k+1} = G + H uhat^k (items: 32-element tiles)
__global__ void __launch_bounds__(32 * kStepT) k_batch_final(const BInst* inst, const int* pre,
                                                             int n_inst, int nmax, int nqmax) {
  extern __shared__ double sm[];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  double* Hsh = sm;                                   // [n][NQFS]
  double* uh = Hsh + nmax * nqmax;                    // [NQFS][32]
  const int n_items = pre[n_inst];
  int cur = -1;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int i = static_owner(pre, n_inst, it);
    const BInst& I = inst[i];
    if (i != cur) {
      __syncthreads();
      for (int k = tid; k < I.n * I.NQFS; k += 32 * kStepT) Hsh[k] = I.H[k];
      cur = i;
    }
    FinalParams p = {};
    p.nel = I.nel;
    p.nface = I.nface;
    p.n = I.n;
    p.NQFS = I.NQFS;
    p.Nqf = I.Nqf;
    p.F = I.F;
    p.shared = 1;
    p.cn = I.cn;
    p.elem_face = I.elem_face;
    p.uhat = I.uhat;
    p.it = I.it;
    p.G = I.G;
    p.H = I.H;
    p.u = I.u;
    const double* src = I.uhat + (int64_t)((I.it->k + 1) & 1) * I.Nqf * I.nface;
    final_tile(p, Hsh, uh, src, it - pre[i]);
  }
}

// the final trace becomes the state's trace in slot 0 (Crank-Nicolson:
// 2 vhat - uhat^n, and the previous-level copies are updated; backward Euler
// reads neither copy, and with K even the final trace is in slot 0 already)
// (items: chunks)
__global__ void __launch_bounds__(256) k_batch_trace_end(const BInst* inst, const int* pre,
                                                         int n_inst) {
  const int n_items = pre[n_inst];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int i = static_owner(pre, n_inst, it);
    const BInst& I = inst[i];
    const int64_t total = (int64_t)I.Nqf * I.nface;
    const int K = I.it->k;
    if (!I.cn && !(K & 1)) continue;
    const double* fin = I.uhat + (int64_t)(K & 1) * total;
    const int64_t t0 = (int64_t)(it - pre[i]) * kApplyChunk;
    const int64_t t1 = std::min<int64_t>(t0 + kApplyChunk, total);
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      if (!I.cn) {
        I.uhat[t] = fin[t];
        continue;
      }
      const double v = 2.0 * fin[t] - I.uhat_n[t];
      I.uhat[t] = v;
      I.uhat_n[t] = v;
      I.gb_old[t] = I.gb[t];
    }
  }
}

// the step's record (iterations, status) and the instance's time: from the
// step's start to its convergence
__global__ void k_batch_end(const BInst* inst, int n_inst, const int* qerr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  const BInst& I = inst[i];
  IterState* it = I.it;
  // the persistent loop gave up a bounded wait: the step did not complete
  if (qerr && *qerr && it->cont) it->status = EHDG_ERR_TIMEOUT;
  const int s = it->step;
  if (s >= 0 && s < I.step_cap) {
    I.step_iters[s] = it->k;
    I.step_status[s] = it->status;
  }
  it->step = s + 1;
  const unsigned long long t = *I.t_conv ? *I.t_conv : global_ns();
  *I.t_acc += t - *I.t_start;
  *I.t_conv = 0ull;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

bool batch_loop_ok(const Ctx& c) {
  const bool nq_ok = c.NQFS == 8 || c.NQFS == 12 || c.NQFS == 16 || c.NQFS == 20 ||
                     c.NQFS == 24 || c.NQFS == 28;
  const bool prec_ok = c.precision == EHDG_FP64 || c.precision == EHDG_MIXED_TF32 ||
                       c.precision == EHDG_MIXED_BF16 || c.precision == EHDG_MIXED_FP32;
  return c.use_pe && !c.use_ozaki && nq_ok && prec_ok &&
         (c.precision == EHDG_FP64 || c.precision == EHDG_MIXED_FP32 || tc_supported(c));
}

// The persistent form applies to these looped instances: every one is FP64 or
// has FP32 corrections, and their largest stages fit the ring together (an
// instance holds at most one stage's items in it at a time) with two
// positions per block (its item and its next claim), at most 8 blocks per SM.
bool batch_persist_fits(const std::vector<const Ctx*>& looped) {
  int64_t need = 0;
  for (const Ctx* c : looped) {
    const bool mma = c->mixed && c->precision != EHDG_MIXED_FP32;
    if (mma) return false;
    const int64_t tiles = (c->nel + kPeTile - 1) / kPeTile;
    const int64_t corr = c->mixed ? (tiles + kQCorrTiles - 1) / kQCorrTiles : 0;
    const int64_t chunks =
        c->mixed ? ((int64_t)c->Nqf * c->nface + kApplyChunk - 1) / kApplyChunk : 0;
    need += std::max({tiles, corr, chunks});
  }
  return need + 16 * (int64_t)device_sms() <= kQCap;
}

struct BatchLoop::Impl {
  BInst* d_inst = nullptr;
  int4* d_counts = nullptr;
  int* d_lists = nullptr;
  unsigned char* d_bimg = nullptr;   // operator images and row tables of the mixed instances
  int* d_pre32 = nullptr;       // static lists: 32-element tiles, trace chunks
  int* d_prech = nullptr;
  int n32 = 0, nch = 0, nmax = 1, nqmax = 1;
  int step_grid = 1, final_grid = 1, chunk_grid = 1;
  size_t step_smem = 0, final_smem = 0;
  unsigned int* d_ticket = nullptr;
  int n_inst = 0, n_sweep = 0, n_tc = 0, n_apply = 0, max_m = 0;
  bool any_mma = false, any_fp32 = false;   // mixed instances with each kind of correction
  int sweep_grid = 1, tc_grid = 1, apply_grid = 1, tc_ncols = 32, tc_smem_b = 0, tc_smem_a = 0;
  int lp_grid = 1;
  size_t lp_smem = 0;
  size_t sweep_smem = 0, tc_smem = 0;
  // persistent form: the work ring and the per-instance stage counters
  BQueue* d_q = nullptr;
  unsigned char* d_rows = nullptr;   // sweep rows in row order of every instance
  long long* d_seq = nullptr;
  int2* d_items = nullptr;
  int* d_stage_cnt = nullptr;
  int persist_grid = 1;
  size_t persist_smem = 0;
};

BatchLoop::~BatchLoop() { release(); }

void BatchLoop::release() {
  if (!impl) return;
  cudaFree(impl->d_inst);
  cudaFree(impl->d_counts);
  cudaFree(impl->d_lists);
  cudaFree(impl->d_pre32);
  cudaFree(impl->d_bimg);
  cudaFree(impl->d_prech);
  cudaFree(impl->d_ticket);
  cudaFree(impl->d_q);
  cudaFree(impl->d_rows);
  cudaFree(impl->d_seq);
  cudaFree(impl->d_items);
  cudaFree(impl->d_stage_cnt);
  delete impl;
  impl = nullptr;
}

// Device tables of the looped instances (their contexts must stay alive).
cudaError_t BatchLoop::build(const std::vector<Ctx*>& ctxs, unsigned long long* t_start,
                             unsigned long long* t_acc, unsigned long long* t_conv,
                             const std::vector<int>& slot) {
  release();
  impl = new Impl();
  Impl& L = *impl;
  L.n_inst = (int)ctxs.size();
  std::vector<BInst> h(L.n_inst);
  std::vector<int4> cnt(L.n_inst);
  std::vector<int> pre32, prech;
  size_t smem = sizeof(int) * 5 * kPeTile;          // the list builder's scan
  int max_kp_bytes = 0, max_np = 16;
  for (int i = 0; i < L.n_inst; ++i) {
    const Ctx& c = *ctxs[i];
    BInst& I = h[i];
    I = BInst{};
    I.nel = c.nel;
    I.nface = c.nface;
    I.NQFS = c.NQFS;
    I.Nqf = c.Nqf;
    I.F = c.F;
    I.n_rows = c.n_rows;
    I.n_up = c.n_up;
    I.n_tiles_pe = (int)((c.nel + kPeTile - 1) / kPeTile);
    I.rows = c.rows;
    I.elem_face = c.geo.elem_face;
    I.face_jf = c.geo.face_jf;
    fill_face_weights(c, I.fw);
    I.Gy = c.Gy;
    I.Y = c.Y;
    I.R_out = c.mixed ? c.R32 : nullptr;
    I.Hy = c.Hy;
    I.uhat = c.uhat;
    I.it = c.it;
    I.partials = c.partials;
    I.hist = c.hist;
    I.tol = c.tol;
    I.res_scale = c.res_scale;
    I.max_iter = c.max_iter;
    I.t_conv = t_conv + slot[i];
    I.t_start = t_start + slot[i];
    I.t_acc = t_acc + slot[i];
    I.err = c.tc_err;
    I.n = c.n;
    I.KE = c.KE;
    I.cn = (c.scheme == EHDG_CN) ? 1 : 0;
    I.ucoef = (c.scheme == EHDG_STEADY) ? 0.0 : 1.0 / c.dt_eff;
    I.P = c.P;
    I.u = c.u;
    I.ey_idx = c.ey_idx;
    I.ey_val = c.ey_val;
    I.G = c.G;
    I.H = c.H;
    I.uhat_n = c.uhat_n;
    I.gb = c.gb;
    I.gb_old = c.gb_old;
    I.sgn = c.sgn;
    I.face_elem = c.geo.face_elem;
    I.face_local = c.geo.face_local;
    I.step_iters = c.step_iters;
    I.step_status = c.step_status;
    I.step_cap = c.step_cap;
    pre32.push_back(L.n32);
    prech.push_back(L.nch);
    L.n32 += (int)((c.nel + 31) / 32);
    L.nch += (int)(((int64_t)c.Nqf * c.nface + kApplyChunk - 1) / kApplyChunk);
    L.nmax = std::max(L.nmax, c.n);
    L.nqmax = std::max(L.nqmax, c.NQFS);
    smem = std::max(smem, sizeof(double) * (size_t)c.n_rows * c.NQFS);
    L.n_sweep += I.n_tiles_pe;
    if (c.mixed) {
      I.tc = 1;
      I.mma = c.precision != EHDG_MIXED_FP32 ? 1 : 0;
      I.bf16 = c.precision == EHDG_MIXED_BF16 ? 1 : 0;
      I.m = c.inner_sweeps;
      I.Hy32 = c.Hy32;
      I.R32 = c.R32;
      I.d32 = c.d32;
      I.Y32 = c.Y32;
      L.max_m = std::max(L.max_m, I.m);
      if (I.mma) {
        const int kstep = I.bf16 ? 16 : 8;
        I.Kp = (c.NQFS + kstep - 1) / kstep * kstep;
        I.Np = std::max(16, (c.n_rows + 15) / 16 * 16);
        I.idesc = umma_idesc(I.bf16 ? 1u : 2u, kBTcM, I.Np);
        // the fixed-shape body where the single-problem sweep runs it
        I.fx = (c.tc_fx && c.F == 4 && c.Nqf >= 2 && c.Nqf <= 7) ? 1 : 0;
        I.nrf = c.tc_nrf;
        I.nupf = c.tc_nupf;
        for (int r = 0; r < 6; ++r) I.rfs[r] = c.tc_rfs[r];
        max_kp_bytes = std::max(max_kp_bytes, I.Kp * (I.bf16 ? 2 : 4));
        max_np = std::max(max_np, I.Np);
        L.any_mma = true;
      } else {
        L.any_fp32 = true;
      }
      I.n_tiles128 = (int)((c.nel + kBTcM - 1) / kBTcM);
      const int64_t total = (int64_t)c.Nqf * c.nface;
      I.n_chunks = (int)((total + kApplyChunk - 1) / kApplyChunk);
      L.n_tc += I.n_tiles128;
      L.n_apply += I.n_chunks;
    }
    cnt[i] = make_int4(I.n_tiles_pe, I.tc, I.n_tiles128, I.n_chunks);
  }
  L.sweep_smem = smem;
  pre32.push_back(L.n32);
  prech.push_back(L.nch);
  cudaError_t e;
  if ((e = cudaMalloc(&L.d_pre32, sizeof(int) * pre32.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.d_prech, sizeof(int) * prech.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpy(L.d_pre32, pre32.data(), sizeof(int) * pre32.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpy(L.d_prech, prech.data(), sizeof(int) * prech.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  const size_t list_ints = kListHeader + 5 * (size_t)L.n_inst + 3;
  // operator images and row tables of the mixed-precision instances
  {
    std::vector<size_t> off(L.n_inst, 0), roff(L.n_inst, 0);
    size_t bytes = 0;
    for (int i = 0; i < L.n_inst; ++i) {
      if (!h[i].mma) continue;
      off[i] = bytes;
      bytes += ((size_t)h[i].Np * h[i].Kp * (h[i].bf16 ? 2 : 4) + 255) / 256 * 256;
      roff[i] = bytes;
      bytes += ((size_t)h[i].Np * sizeof(int) + 255) / 256 * 256;
    }
    if (bytes > 0) {
      if ((e = cudaMalloc(&L.d_bimg, bytes)) != cudaSuccess) return e;
      for (int i = 0; i < L.n_inst; ++i) {
        if (!h[i].mma) continue;
        const Ctx& c = *ctxs[i];
        k_batch_bimg<<<1, 256>>>(c.Hy32, c.rows, c.n_rows, c.NQFS, c.Nqf, h[i].Np, h[i].Kp,
                                 h[i].bf16, L.d_bimg + off[i],
                                 reinterpret_cast<int*>(L.d_bimg + roff[i]));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        h[i].Bimg = reinterpret_cast<const uint4*>(L.d_bimg + off[i]);
        h[i].rowfg = reinterpret_cast<const int*>(L.d_bimg + roff[i]);
      }
      if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    }
  }
  const bool persist_fits =
      batch_persist_fits(std::vector<const Ctx*>(ctxs.begin(), ctxs.end()));
  if (!L.any_mma && persist_fits) {
    // the persistent form reads every instance's sweep rows in row order
    std::vector<size_t> off(L.n_inst, 0), off32(L.n_inst, 0);
    size_t bytes = 0;
    for (int i = 0; i < L.n_inst; ++i) {
      off[i] = bytes;
      bytes += (sizeof(double) * h[i].n_rows * h[i].NQFS + 255) / 256 * 256;
      off32[i] = bytes;
      if (h[i].tc) bytes += (sizeof(float) * h[i].n_rows * h[i].NQFS + 255) / 256 * 256;
    }
    if ((e = cudaMalloc(&L.d_rows, std::max<size_t>(bytes, 256))) != cudaSuccess) return e;
    for (int i = 0; i < L.n_inst; ++i) {
      const Ctx& c = *ctxs[i];
      double* hyc = reinterpret_cast<double*>(L.d_rows + off[i]);
      float* hy32c = h[i].tc ? reinterpret_cast<float*>(L.d_rows + off32[i]) : nullptr;
      k_batch_rows<<<1, 256>>>(c.Hy, h[i].tc ? c.Hy32 : nullptr, c.rows, c.n_rows, h[i].n_up,
                               c.NQFS, hyc, hy32c);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      h[i].Hyc = hyc;
      h[i].Hy32c = hy32c;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
  }
  if ((e = cudaMalloc(&L.d_inst, sizeof(BInst) * std::max(1, L.n_inst))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.d_counts, sizeof(int4) * std::max(1, L.n_inst))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(L.d_counts, cnt.data(), sizeof(int4) * L.n_inst, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMalloc(&L.d_lists, sizeof(int) * list_ints)) != cudaSuccess) return e;
  if ((e = cudaMemset(L.d_lists, 0, sizeof(int) * list_ints)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.d_ticket, sizeof(unsigned int))) != cudaSuccess) return e;
  if ((e = cudaMemset(L.d_ticket, 0, sizeof(unsigned int))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(L.d_inst, h.data(), sizeof(BInst) * L.n_inst, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  // launch shapes: one wave of resident blocks each, capped by the most work
  // an iteration can have (every instance iterating)
  auto wave = [](auto kernel, int threads, size_t sm, int items) {
    int bpsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, kernel, threads, sm) != cudaSuccess ||
        bpsm < 1) {
      cudaGetLastError();
      bpsm = 1;
    }
    return std::max(1, std::min(bpsm * device_sms(), items));
  };
  L.sweep_grid = wave(k_batch_sweep, kPeTile, smem, L.n_sweep);
  L.step_smem = sizeof(double) * ((size_t)L.nmax * L.nmax + 64 * (size_t)L.nmax);
  L.final_smem = sizeof(double) * ((size_t)L.nmax * L.nqmax + 32 * (size_t)L.nqmax);
  if ((e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)L.step_smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_batch_final, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)L.final_smem)) != cudaSuccess)
    return e;
  L.step_grid = wave(k_batch_step, 32 * kStepT, L.step_smem, L.n32);
  L.final_grid = wave(k_batch_final, 32 * kStepT, L.final_smem, L.n32);
  L.chunk_grid = std::max(1, std::min(device_sms() * 8, L.nch));
  if (L.any_fp32) {
    for (int i = 0; i < L.n_inst; ++i)
      if (h[i].tc && !h[i].mma)
        L.lp_smem = std::max(L.lp_smem, sizeof(float) * (size_t)h[i].n_up * h[i].NQFS);
    L.lp_grid = wave(k_batch_lp, kPeTile, L.lp_smem, L.n_tc);
    L.apply_grid = std::max(1, std::min(device_sms() * 8, L.n_apply));
  }
  if (L.any_mma) {
    // B: the largest instance's padded rows x K; A: 128 x K
    L.tc_smem_b = (max_np * max_kp_bytes + 1023) / 1024 * 1024;
    L.tc_smem_a = (kBTcM * max_kp_bytes + 15) / 16 * 16;
    L.tc_smem = (size_t)L.tc_smem_b + L.tc_smem_a + sizeof(int) * (6 * kBTcM + 512) + 1024;
    while (L.tc_ncols < max_np) L.tc_ncols *= 2;
    if ((e = cudaFuncSetAttribute(k_batch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.tc_smem)) != cudaSuccess)
      return e;
    int bpsm = (int)((227 * 1024) / (L.tc_smem + 1024));
    bpsm = std::max(1, std::min({bpsm, 512 / L.tc_ncols, 8}));
    L.tc_grid = std::max(1, std::min(bpsm * device_sms(), L.n_tc));
    L.apply_grid = std::max(1, std::min(device_sms() * 8, L.n_apply));
  }
  if (!L.any_mma && persist_fits) {
    // the persistent form: one wave of resident blocks
    if ((e = cudaMalloc(&L.d_q, sizeof(BQueue))) != cudaSuccess) return e;
    if ((e = cudaMemset(L.d_q, 0, sizeof(BQueue))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&L.d_seq, sizeof(long long) * kQCap)) != cudaSuccess) return e;
    if ((e = cudaMemset(L.d_seq, 0xFF, sizeof(long long) * kQCap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&L.d_items, sizeof(int2) * kQCap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&L.d_stage_cnt, sizeof(int) * std::max(1, L.n_inst))) != cudaSuccess)
      return e;
    // the operator rows come from global memory: no dynamic shared memory
    L.persist_smem = 0;
    L.persist_grid = wave(k_batch_persist, kPeTile, L.persist_smem, 1 << 30);
  }
  return cudaSuccess;
}

bool BatchLoop::persist_ok() const { return impl && impl->d_q; }

// The persistent loop of a step (after launch_pre with graph_mode 0): the
// ring's start, then one launch that runs every remaining iteration.
cudaError_t BatchLoop::launch_persist(cudaStream_t s) {
  Impl& L = *impl;
  k_batch_qinit<<<1, 256, 0, s>>>(L.d_inst, L.n_inst, L.d_q, L.d_seq, L.d_items, L.d_stage_cnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_batch_persist<<<L.persist_grid, kPeTile, L.persist_smem, s>>>(
      L.d_inst, L.d_q, L.d_seq, L.d_items, L.d_stage_cnt, kQWaitLimit);
  return cudaGetLastError();
}

// Self-test of the ring's bounded wait: one live instance and nothing ever
// published, so every block polls an empty slot, gives up after `limit` polls
// and leaves; *gave_up receives the ring's error flag (1 as designed).
cudaError_t batch_ring_selftest(cudaStream_t s, unsigned int limit, int* gave_up) {
  BQueue* q = nullptr;
  long long* seq = nullptr;
  int2* items = nullptr;
  int* cnt = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(BQueue));
  if (e == cudaSuccess) e = cudaMalloc(&seq, sizeof(long long) * kQCap);
  if (e == cudaSuccess) e = cudaMalloc(&items, sizeof(int2) * kQCap);
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int));
  BQueue h{};
  h.live = 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(q, &h, sizeof(BQueue), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(seq, 0xFF, sizeof(long long) * kQCap, s);
  if (e == cudaSuccess) {
    k_batch_persist<<<2, kPeTile, 0, s>>>(nullptr, q, seq, items, cnt, limit);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, q, sizeof(BQueue), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *gave_up = h.err;
  cudaFree(q);
  cudaFree(seq);
  cudaFree(items);
  cudaFree(cnt);
  return e;
}

// Everything of a step before the loop, each kernel one launch for all the
// looped instances: reset and start time, right-hand side, initial trace,
// the work lists, and the first FP64 sweep (which sets the loop condition).
cudaError_t BatchLoop::launch_pre(cudaStream_t s, cudaGraphConditionalHandle handle,
                                  int graph_mode) {
  Impl& L = *impl;
  cudaError_t e;
  k_batch_begin<<<(L.n_inst + 127) / 128, 128, 0, s>>>(L.d_inst, L.n_inst);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_batch_step<<<L.step_grid, dim3(32, kStepT), L.step_smem, s>>>(L.d_inst, L.d_pre32, L.n_inst,
                                                                  L.nmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_batch_trace0<<<L.chunk_grid, 256, 0, s>>>(L.d_inst, L.d_prech, L.n_inst);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_batch_lists<<<1, 256, sizeof(int) * 5 * 256, s>>>(L.d_inst, L.d_counts, L.n_inst,
                                                       L.d_lists);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_batch_sweep<<<L.sweep_grid, kPeTile, L.sweep_smem, s>>>(L.d_inst, L.d_counts, L.d_lists,
                                                           L.n_inst, L.d_ticket, graph_mode,
                                                           handle);
  return cudaGetLastError();
}

// Everything of a step after the loop: reconstruction, trace hand-over,
// step record and instance times.
cudaError_t BatchLoop::launch_post(cudaStream_t s) {
  Impl& L = *impl;
  cudaError_t e;
  k_batch_final<<<L.final_grid, dim3(32, kStepT), L.final_smem, s>>>(L.d_inst, L.d_pre32,
                                                                    L.n_inst, L.nmax, L.nqmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_batch_trace_end<<<L.chunk_grid, 256, 0, s>>>(L.d_inst, L.d_prech, L.n_inst);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_batch_end<<<(L.n_inst + 127) / 128, 128, 0, s>>>(L.d_inst, L.n_inst,
                                                     L.d_q ? &L.d_q->err : nullptr);
  return cudaGetLastError();
}

// The loop body (captured into the WHILE node's body graph on stream s).
cudaError_t BatchLoop::launch_body(cudaStream_t s, cudaGraphConditionalHandle handle) {
  Impl& L = *impl;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < L.max_m && L.n_tc; ++j) {
    if (L.any_mma) {
      k_batch_tc<<<L.tc_grid, kBTcThreads, L.tc_smem, s>>>(L.d_inst, L.d_lists, L.n_inst, j,
                                                          L.tc_ncols, L.tc_smem_b, L.tc_smem_a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (L.any_fp32) {
      k_batch_lp<<<L.lp_grid, kPeTile, L.lp_smem, s>>>(L.d_inst, L.d_lists, L.n_inst, j);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  if (L.n_apply) {
    k_batch_apply<<<L.apply_grid, 256, 0, s>>>(L.d_inst, L.d_lists, L.n_inst);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_batch_sweep<<<L.sweep_grid, kPeTile, L.sweep_smem, s>>>(L.d_inst, L.d_counts, L.d_lists,
                                                           L.n_inst, L.d_ticket, 1, handle);
  return cudaGetLastError();
}

// One step of the looped instances driven from the host, every launch
// bracketed by CUDA events on stream s (kernel accounting): the same kernels
// as the graph, the loop condition read back after every iteration.
cudaError_t BatchLoop::run_step_profiled(cudaStream_t s, int max_iter, double* ms,
                                         int64_t* launches, bool persist) {
  Impl& L = *impl;
  cudaEvent_t ev[2];
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  auto timed = [&](int kind, auto&& launch) -> cudaError_t {
    cudaError_t r = cudaEventRecord(ev[0], s);
    if (r == cudaSuccess) r = launch();
    if (r == cudaSuccess) r = cudaEventRecord(ev[1], s);
    if (r == cudaSuccess) r = cudaEventSynchronize(ev[1]);
    float t = 0.f;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&t, ev[0], ev[1]);
    ms[kind] += t;
    launches[kind] += 1;
    return r;
  };
  const cudaGraphConditionalHandle none = 0;
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_AUX, [&] {
    k_batch_begin<<<(L.n_inst + 127) / 128, 128, 0, s>>>(L.d_inst, L.n_inst);
    return cudaGetLastError();
  });
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_STEP, [&] {
    k_batch_step<<<L.step_grid, dim3(32, kStepT), L.step_smem, s>>>(L.d_inst, L.d_pre32,
                                                                    L.n_inst, L.nmax);
    return cudaGetLastError();
  });
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_FACE, [&] {
    k_batch_trace0<<<L.chunk_grid, 256, 0, s>>>(L.d_inst, L.d_prech, L.n_inst);
    return cudaGetLastError();
  });
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_AUX, [&] {
    k_batch_lists<<<1, 256, sizeof(int) * 5 * 256, s>>>(L.d_inst, L.d_counts, L.n_inst,
                                                         L.d_lists);
    return cudaGetLastError();
  });
  auto sweep = [&] {
    return timed(EHDG_KERNEL_ELEM, [&] {
      k_batch_sweep<<<L.sweep_grid, kPeTile, L.sweep_smem, s>>>(
          L.d_inst, L.d_counts, L.d_lists, L.n_inst, L.d_ticket, 0, none);
      return cudaGetLastError();
    });
  };
  if (e == cudaSuccess) e = sweep();
  if (persist && persist_ok()) {
    // every remaining iteration in the persistent launch (timed as ELEM)
    if (e == cudaSuccess) e = timed(EHDG_KERNEL_ELEM, [&] { return launch_persist(s); });
    max_iter = 0;
  }
  int n_active = 0;
  for (int it = 0; e == cudaSuccess && it < max_iter; ++it) {
    if ((e = cudaMemcpy(&n_active, L.d_lists, sizeof(int), cudaMemcpyDeviceToHost)) !=
        cudaSuccess || n_active == 0)
      break;
    for (int j = 0; j < L.max_m && L.n_tc && e == cudaSuccess; ++j) {
      if (L.any_mma)
        e = timed(EHDG_KERNEL_CORR, [&] {
          k_batch_tc<<<L.tc_grid, kBTcThreads, L.tc_smem, s>>>(L.d_inst, L.d_lists, L.n_inst,
                                                              j, L.tc_ncols, L.tc_smem_b,
                                                              L.tc_smem_a);
          return cudaGetLastError();
        });
      if (L.any_fp32 && e == cudaSuccess)
        e = timed(EHDG_KERNEL_CORR, [&] {
          k_batch_lp<<<L.lp_grid, kPeTile, L.lp_smem, s>>>(L.d_inst, L.d_lists, L.n_inst, j);
          return cudaGetLastError();
        });
    }
    if (L.n_apply && e == cudaSuccess)
      e = timed(EHDG_KERNEL_AUX, [&] {
        k_batch_apply<<<L.apply_grid, 256, 0, s>>>(L.d_inst, L.d_lists, L.n_inst);
        return cudaGetLastError();
      });
    if (e == cudaSuccess) e = sweep();
  }
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_FINAL, [&] {
    k_batch_final<<<L.final_grid, dim3(32, kStepT), L.final_smem, s>>>(
        L.d_inst, L.d_pre32, L.n_inst, L.nmax, L.nqmax);
    return cudaGetLastError();
  });
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_FACE, [&] {
    k_batch_trace_end<<<L.chunk_grid, 256, 0, s>>>(L.d_inst, L.d_prech, L.n_inst);
    return cudaGetLastError();
  });
  if (e == cudaSuccess) e = timed(EHDG_KERNEL_AUX, [&] {
    k_batch_end<<<(L.n_inst + 127) / 128, 128, 0, s>>>(L.d_inst, L.n_inst,
                                                       L.d_q ? &L.d_q->err : nullptr);
    return cudaGetLastError();
  });
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return e;
}

int BatchLoop::kernels_per_iteration() const {
  return impl ? (impl->n_tc ? impl->max_m : 0) + (impl->n_apply ? 1 : 0) + 1 : 0;
}

}  // namespace ehdg
