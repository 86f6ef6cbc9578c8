// Internal declarations of libehdg: context, reference tables, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/ehdg.h"

namespace ehdg {

// ---------------------------------------------------------------------------
// 1D reference tables (host side, built independently of any other code)
// ---------------------------------------------------------------------------
struct Ref1D {
  int p = 0, q = 0;
  std::vector<double> r, wr;      // GLL nodes and weights (p+1)
  std::vector<double> xi, om;     // Gauss points and weights (q)
  std::vector<double> L, D;       // [q][p+1] l_a(xi_g), l_a'(xi_g)
  std::vector<double> Lend;       // [2][p+1] l_a(-1), l_a(+1)
};
void build_ref1d(int p, int q, Ref1D* out);
void gll_rule(int p, std::vector<double>* x, std::vector<double>* w);
void gauss_rule(int q, std::vector<double>* x, std::vector<double>* w);

// ---------------------------------------------------------------------------
// Device-side problem description handed to kernels (by value)
// ---------------------------------------------------------------------------
constexpr int kMaxP1 = 10;        // max points per axis in the 1D tables
constexpr int kMaxQ = 10;

struct RefTables {               // lives in kernel parameter space (small)
  int dim, p, q, Np, Nqf, nf;
  double L[kMaxQ * kMaxP1];
  double D[kMaxQ * kMaxP1];
  double Lend[2 * kMaxP1];
  double om[kMaxQ];
  double xi[kMaxQ];               // Gauss points on [-1, 1]
};

struct Geometry {
  int64_t nel, nface;
  const double* elem_h;          // [nel][dim]
  const int32_t* elem_face;      // SoA [2*dim][nel]
  const int32_t* face_elem;      // SoA [2][nface]
  const int8_t* face_local;      // SoA [2][nface]
  const int8_t* face_tag;        // [nface]
  const double* face_jf;         // [nface] face Jacobian J_f
};

// Iteration state word kept on the device (one per context).
struct IterState {
  int k;                         // iterations done in the current step
  int cont;                      // 1 while the loop must go on
  int status;                    // ehdg_status of the current step
  unsigned int counter;          // last-block ticket of the residual reduction
  int step;                      // steps finished since the last reset (ehdg_run)
  unsigned int bar;              // grid-barrier arrivals of a persistent sweep
  int abort;                     // a persistent sweep's bounded wait gave up
  double r_last;
};

struct Ctx {
  // problem
  int dim = 0, p = 0, nf = 1, Np = 0, n = 0, q = 0, Nqf = 0, F = 0, NQFS = 0;
  int64_t nel = 0, nface = 0;
  ehdg_pde pde = EHDG_TRANSPORT;
  ehdg_scheme scheme = EHDG_BE;
  double dt = 0, dt_eff = 0, tol = 0, Phi = 1, res_scale = 1;
  double cor_f0 = 0, cor_beta = 0, cor_ym = 0, friction = 0;   // shallow-water source terms
  int max_iter = 0;
  bool shared_op = false;        // one operator for all elements
  bool variable_beta = false;
  double beta_const[3] = {0, 0, 0};
  uint64_t beta_nodes_hash = 0;  // FNV-1a of the nodal velocity (variable case), for checkpoints
  cudaStream_t stream = nullptr;
  RefTables ref{};
  Ref1D r1d;
  int KE = 0;                    // nonzeros per row of the face-point extraction

  // host copies for coordinates
  std::vector<double> elem_lo, elem_h;
  std::vector<int64_t> face_elem_h, elem_face_h;
  std::vector<int8_t> face_local_h;

  // device memory
  std::vector<void*> allocs;
  int64_t bytes = 0;
  Geometry geo{};
  double* beta_nodes = nullptr;  // [nel][dim][Np] (variable velocity)
  double* elem_lo_d = nullptr;   // [nel][dim] element lower corners (beta-plane Coriolis)
  double* P = nullptr;           // [n][n][ne]   A^{-1} Mblk
  double* H = nullptr;           // [n][NQFS][ne] A^{-1} B
  double* Hy = nullptr;          // [NQFS][NQFS][ne] face-point rows of H
  int* ey_idx = nullptr;         // [NQFS][KE]
  double* ey_val = nullptr;      // [NQFS][KE]
  int8_t* sgn = nullptr;         // [Nqf][nface] sgn(beta.n^-) (transport)
  int* rows = nullptr;           // shared operator: element output rows (face points)
  int n_rows = 0;
  std::vector<int> rows_host;    // host copy of rows
  uint8_t* rowid = nullptr;      // per-element operator: [NQFS][nel] row of each slot
  uint8_t* nrows = nullptr;      // [nel] slots in use
  uint8_t* nup = nullptr;        // [nel] leading slots that are upwind points (transport)
  int n_up = 0;                  // shared operator: leading upwind rows
  int32_t* tan_g = nullptr;      // face points with beta.n = 0: point index
  int32_t* tan_face = nullptr;   //   and face
  int64_t n_tan = 0;
  int64_t sweep_rows = 0;        // rows computed per sweep, all elements
  // per-element transport operator, tile-major (32 elements per tile): the
  // rows each tile needs, NQFS x 32 doubles each, streamed by the tiled sweep
  double* Hyt = nullptr;
  int32_t* tile_row0 = nullptr;  // [ntiles] first row of a tile in Hyt
  uint8_t* tile_nrows = nullptr; // [ntiles] rows of a tile (max over its elements)
  int64_t ntiles = 0;
  int64_t tile_rows = 0;         // rows in Hyt
  int tiled_grid = 0;            // launch shape of the tiled sweep
  size_t tiled_smem = 0;
  int32_t* tiled_warp_tile = nullptr;   // [tiled_grid * warps per block] first tile of a warp
  double* Ht = nullptr;          // reconstruction operator H, tile-major: [tile][n][NQFS][32]
  float* Hyt32 = nullptr;        // FP32 copy of Hyt (mixed precision, FP32)
  void* Hyt16 = nullptr;         // BF16 copy of Hyt (mixed precision, BF16)
  int32_t* ptid = nullptr;       // [slot][nel] trace index of each row's point (mixed)
  int lp_grid = 0;               // launch shape of the tiled correction sweep
  size_t lp_smem = 0;
  int32_t* lp_warp_tile = nullptr;   // [lp_grid * warps per block] first tile of a warp
  int ftiled_grid = 0;           // launch shape of the tiled reconstruction
  size_t ftiled_smem = 0;
  bool persist_fits = false;     // the persistent sweep's grid is co-resident
  double* ppartials = nullptr;   // [2][tiled_grid] its residual partials
  // mixed precision (defect correction)
  bool mixed = false;
  ehdg_precision precision = EHDG_FP64;
  int* tc_err = nullptr;         // set by a sweep whose bounded mbarrier wait gave up
  // tensor-core correction sweep (TF32/BF16, shared operator): the sweep rows
  // rounded into the K-major shared-memory image at setup and, for the
  // fixed-shape form (rows are whole faces), the local face of each row face
  void* tc_img = nullptr;
  bool tc_fx = false;
  int32_t* bface = nullptr;      // [n_bface] boundary faces (ascending)
  int64_t n_bface = 0;
  int tc_nrf = 0, tc_nupf = 0;   // row faces; leading ones owned (upwind)
  int tc_rfs[6] = {0, 0, 0, 0, 0, 0};
  // FP64-accurate products on the BF16 tensor cores (Ozaki splitting, shared
  // operator): the sweep (Hy rows), the reconstruction (H) and the step (P)
  bool use_ozaki = false;
  int path_gen = 0;              // bumped when the FP64 path is switched (captured graphs go stale)
  struct OzOp {
    void* img = nullptr;         // [7 * LS x KP] BF16 digit slices of the operator rows
    int* Fb = nullptr;           // [LS] largest biased exponent of each row
    int rows = 0, Np = 0, LS = 0, ncols = 0, KP = 0, tpe = 0;   // rows, padded, TMEM, K
    int grid = 0, threads = 0;
    size_t smem = 0;
  } oz_sweep, oz_final, oz_step;
  // sum-factorised FP64 sweep and reconstruction (hexahedra, one shared
  // transport operator): the element's face traces go to its boundary nodes
  // by two 1D passes per face (Bs), then Dy = Ey A^{-1}[:, bnd] gives the
  // face-point rows and Ab = A^{-1}[:, bnd] the volume values
  bool use_pe = false;           // 2D shared-operator FP64 sweep, one thread per element
  double* pe_fw = nullptr;       // its face Gauss weights [Nqf]
  bool use_sf = false;
  int sf_NB = 0;                 // boundary nodes per element
  int* sf_bnd = nullptr;         // [NB] their node indices
  double* sf_Ab = nullptr;       // [n][NB]
  double* sf_Dy = nullptr;       // [NQFS][NB]
  double sf_s[6] = {0, 0, 0, 0, 0, 0};   // J_f |beta.n| of each local face
  std::vector<int> sf_map;       // [NB][3] faces of each boundary node: f | a_t1 << 4 | a_t2 << 8
  int inner_sweeps = 0;
  int sweep_ft = 4;              // row groups per 32-element tile of k_sweep_fused (2, 4 or 8)
  float* Hy32 = nullptr;         // FP32 copy of Hy in the sweep's slot layout
  float* R32 = nullptr;          // [Nqf][nface] FP64 residual F(uhat) - uhat, rounded
  float* d32 = nullptr;          // [2][Nqf][nface] correction iterates
  float* Y32 = nullptr;          // [NQFS][nel] low-precision element values
  double* u = nullptr;           // [n][nel] state u^n (SoA)
  double* G = nullptr;           // [n][nel]
  double* Gy = nullptr;          // [NQFS][nel]
  double* Y = nullptr;           // [NQFS][nel] element values at face points
  double* uhat = nullptr;        // [2][Nqf][nface] trace ping-pong pair; slot 0 holds the state's trace
  double* uhat_n = nullptr;      // [Nqf][nface] trace of the previous step (CN)
  double* gb = nullptr;          // [Nqf][nface] boundary data, new level
  double* gb_old = nullptr;      // [Nqf][nface] boundary data, previous level
  double* force = nullptr;       // [n][nel] forcing (or null)
  double* force_old = nullptr;
  bool have_force = false;
  double* partials = nullptr;    // residual block partials
  int n_partials = 0;
  IterState* it = nullptr;
  // Warm start of the initial trace (backward Euler / steady transport on
  // hexahedra without beta.n = 0 points): *warm = 1 on the device while slot 0
  // of uhat holds the previous step's final trace uhat^K and u the
  // reconstruction from uhat^{K-1}. The last sweep wrote uhat^K = Ey u at every
  // owned point, which is the trace formula of u^n there, so the next step
  // starts from slot 0 and recomputes only the inflow boundary points from the
  // new boundary data, and the step kernel skips Y0 = Ey u^n.
  int* warm = nullptr;           // [1] device flag (part of the saved state)
  bool warm_ok = false;          // this context qualifies
  double* hist = nullptr;        // [max_iter]
  double* staging = nullptr;     // [max(state,trace)] transposition buffer
  IterState* it_host = nullptr;  // pinned
  int last_iters = 0;
  cudaGraphConditionalHandle handle = 0;
  // one implicit step as a CUDA graph: step RHS, initial trace, WHILE{sweep, trace}, end of step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_persist = false;    // the captured step uses the persistent sweep
  bool graph_force = false;      // have_force value the graph was captured with
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
  int* step_iters = nullptr;     // [step_cap] iterations of each step of ehdg_run
  int* step_status = nullptr;
  int step_cap = 0;
  std::vector<int> step_iters_h, step_status_h;

  // kernel accounting (ehdg_set_profiling / ehdg_kernel_stats)
  bool profiling = false;
  int64_t launches[EHDG_KERNEL_KINDS] = {0};
  struct EvRec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<EvRec> ev_used;
  std::vector<cudaEvent_t> ev_pool;
};

// launchers (kernels.cu)
cudaError_t launch_assemble(Ctx& c, int n_assemble);
cudaError_t launch_face_signs(Ctx& c);
cudaError_t launch_step(Ctx& c);
cudaError_t launch_elem(Ctx& c);
cudaError_t launch_face(Ctx& c, int mode, int graph_mode = 0);   // 0 initial trace, 1 iteration
cudaError_t launch_final(Ctx& c);
cudaError_t launch_aos_to_soa(const double* src, double* dst, int64_t outer, int inner,
                              cudaStream_t s);   // src [outer][inner] -> dst [inner][outer]
cudaError_t launch_soa_to_aos(const double* src, double* dst, int64_t outer, int inner,
                              cudaStream_t s);
cudaError_t launch_reset_iter(Ctx& c);
cudaError_t launch_extract(Ctx& c);
cudaError_t launch_step_end(Ctx& c);
cudaError_t launch_stamp(cudaStream_t s, unsigned long long* t_start, unsigned long long* t_acc,
                         int i, int end);
cudaError_t launch_rows(Ctx& c);
int face_grid_x(int64_t nface, int Nqf);   // blocks along faces of the trace kernel
size_t asm_smem(const Ctx& c);     // shared memory of the assembly kernel
// sum-factorised transport sweep and reconstruction (sweep_sf.cu)
bool sf_supported(const Ctx& c);
ehdg_status sf_prepare(Ctx& c);                           // host tables, before assembly
cudaError_t launch_sweep_sf(Ctx& c, int graph_mode, int* grid_out);
cudaError_t launch_final_sf(Ctx& c);
// one-thread-per-element 2D transport sweep (sweep_pe.cu)
bool pe_supported(const Ctx& c);
cudaError_t launch_sweep_pe(Ctx& c, int graph_mode, int* grid_out);
cudaError_t launch_lp_sweep_pe(Ctx& c, const float* in, float* out);   // FP32 corrections
// fused transport sweep (sweep_fused.cu)
cudaError_t launch_sweep_fused(Ctx& c, int graph_mode);
size_t fused_sweep_smem(const Ctx& c);   // dynamic shared memory of the fused sweep
int fused_sweep_grid(const Ctx& c);      // its grid = its residual partials
int fused_grid(int64_t nel);      // upper bound of the fused sweep's grid
int device_sms();
// cached per kernel (and device): raise the dynamic shared-memory limit, set
// the shared-memory carveout to 100, resident blocks per SM
cudaError_t fn_smem(const void* fn, size_t bytes);
cudaError_t fn_carveout(const void* fn);
int fn_blocks_per_sm(const void* fn, int threads, size_t smem);
// resident blocks per SM from the kernel's attributes and the device limits (0 on error)
int fn_blocks_from_attrs(const void* fn, int threads, size_t smem);
int tangent_grid(int64_t n_tan);
void fill_face_weights(const Ctx& c, double* fw);   // face Gauss weight of each face point
// tiled per-element transport sweep (sweep_tiled.cu)
bool tiled_supported(const Ctx& c);
cudaError_t tiled_sweep_shape(const Ctx& c, int64_t rows, int64_t ntiles, int* grid,
                              size_t* smem);             // launch shape of the tiled sweep
cudaError_t build_tiled_operator(Ctx& c);           // after launch_rows; synchronous
cudaError_t launch_sweep_tiled(Ctx& c, int graph_mode, int* grid_out);
int tiled_persist_blocks_per_sm(const Ctx& c);      // co-resident blocks of the persistent sweep
bool persistent_sweep_ok(const Ctx& c);             // whole-step sweep in one launch applies
cudaError_t launch_sweep_persistent(Ctx& c);        // all iterations of a step, one launch
cudaError_t launch_final_tiled(Ctx& c);              // u = G + H uhat, per-element H
cudaError_t launch_lp_sweep_tiled(Ctx& c, const float* in, float* out);   // FP32 correction sweep
// mixed precision (mixed.cu)
cudaError_t launch_hy_to_f32(Ctx& c);
cudaError_t launch_correction(Ctx& c);                    // m inner sweeps + FP64 update
// one inner sweep; fuse_apply: the last one also makes the FP64 update (only
// where tc_apply_fusable; the caller then launches no separate update)
cudaError_t launch_lp_sweep(Ctx& c, const float* in, float* out, bool fuse_apply = false);
cudaError_t launch_apply(Ctx& c, const float* delta);       // uhat += delta in FP64
float* correction_out(Ctx& c, int j);                       // output buffer of inner sweep j
int lp_sweep_launches(const Ctx& c);                        // kernels of one inner sweep
// FP64-accurate tensor-core sweep (ozaki_sweep.cu)
bool ozaki_supported(const Ctx& c);
cudaError_t build_ozaki_operator(Ctx& c);   // after assembly and rows
cudaError_t launch_sweep_ozaki(Ctx& c, int graph_mode, int* grid_out);
cudaError_t launch_elem_ozaki(Ctx& c);      // shallow water: Y = Gy + Hy uhat
cudaError_t launch_final_ozaki(Ctx& c);     // u = G + H uhat (Crank-Nicolson: 2 v - u^n)
cudaError_t launch_step_ozaki(Ctx& c);      // G = P w
cudaError_t dalloc_raw(Ctx& c, void** p, size_t bytes);   // device allocation owned by c
// the device arrays of a context's stepping state (checkpoints, autotuner snapshots)
std::vector<std::pair<void*, size_t>> state_arrays(Ctx& c);
// tensor-core correction sweep (tc_sweep.cu)
bool tc_supported(const Ctx& c);
cudaError_t launch_gather_boundary(const Ctx& c, const double* src, double* dst);
cudaError_t build_tc_image(Ctx& c);   // after the FP32 operator copy
// fuse_apply (only where tc_apply_fusable): the last inner sweep applies the
// correction to uhat in FP64 at the owned points instead of storing it
cudaError_t launch_lp_sweep_tc(Ctx& c, const float* in, float* out, bool fuse_apply = false);
bool tc_apply_fusable(const Ctx& c);

// Batched iteration loop of a batch's looped instances (batch_loop.cu): one
// launch per kernel and iteration over every unconverged instance.
bool batch_loop_ok(const Ctx& c);   // the instance can run in the batched loop
// the batched loop's persistent form applies to these looped instances
bool batch_persist_fits(const std::vector<const Ctx*>& looped);
struct BatchLoop {
  struct Impl;
  Impl* impl = nullptr;
  BatchLoop() = default;
  BatchLoop(const BatchLoop&) = delete;
  BatchLoop& operator=(const BatchLoop&) = delete;
  ~BatchLoop();
  void release();
  // device tables of the looped instances; t_start/t_acc/t_conv[slot[i]]:
  // instance i's step start, accumulated step times and convergence time
  cudaError_t build(const std::vector<Ctx*>& ctxs, unsigned long long* t_start,
                    unsigned long long* t_acc, unsigned long long* t_conv,
                    const std::vector<int>& slot);
  // a step's kernels before the loop (they set the loop condition), the loop
  // body, and the kernels after it
  // (graph_mode 0: the pre-loop sweep sets no conditional handle)
  cudaError_t launch_pre(cudaStream_t s, cudaGraphConditionalHandle handle, int graph_mode = 1);
  cudaError_t launch_body(cudaStream_t s, cudaGraphConditionalHandle handle);
  cudaError_t launch_post(cudaStream_t s);
  // the persistent form of the loop (every remaining iteration of a step in
  // one launch, instances at their own pace), where every looped instance is
  // FP64 or has FP32 corrections
  bool persist_ok() const;
  cudaError_t launch_persist(cudaStream_t s);
  // one step driven from the host, each launch timed with CUDA events:
  // ms[kind] and launches[kind] accumulate (ehdg_kernel_kind)
  cudaError_t run_step_profiled(cudaStream_t s, int max_iter, double* ms, int64_t* launches,
                                bool persist = false);
  int kernels_per_iteration() const;
};

enum FaceMode { kFaceInitial = 0, kFaceIterate = 1 };
int face_launches(const Ctx& c, int mode);   // kernels one launch_face(c, mode) makes
// the persistent batched loop's ring wait against a ring where nothing is ever
// published (ehdg_selftest_wait_timeout, which = 2)
cudaError_t batch_ring_selftest(cudaStream_t s, unsigned int limit, int* gave_up);

void set_last_error(const std::string& msg);
// standalone weighted difference norm (residual.cu); its grid never exceeds
// kResidMaxBlocks blocks, one partial sum each
constexpr int kResidMaxBlocks = 1024;
// standalone weighted difference norm (residual.cu)
cudaError_t launch_wdiff_norm(const double* a, const double* b, const double* w, int64_t n,
                              double* partials, unsigned int* counter, double* out,
                              cudaStream_t s);
int wdiff_norm_blocks(int64_t n);

}  // namespace ehdg

struct ehdg_ctx_s {
  ehdg::Ctx c;
};
