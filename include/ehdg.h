/*
 * ehdg.h -- C ABI of the GB300 eHDG library (libehdg.so).
 *
 * The library runs the eHDG iteration of Muralikrishnan, Tran and Bui-Thanh,
 * "An iterative solver for HDG discretizations of hyperbolic PDEs"
 * (arXiv 1601.06681), Algorithm 1, on one GPU: every iteration solves every
 * element's upwind-HDG local equation for its volume unknowns given the
 * current traces (Sec. 3, eq. transportLocalk1 for transport, eq.
 * localSolverDD for linearised shallow water), then recomputes every face's
 * trace from its two neighbours with the trace formula (Sec. 3, eq.
 * transportLocale, and the shallow-water trace phihat = {{phi}} +
 * sqrt(Phi) {{vel.n}}), and stops on a residual tolerance; one such solve
 * runs inside every implicit time step.
 *
 * Conventions shared by every call:
 *  - Every function returns an ehdg_status; none aborts, traps or exits.
 *    On failure ehdg_last_error() (thread-local) describes the cause.
 *  - The caller owns every pointer it passes. The library copies what it
 *    needs during the call and owns all device memory it allocates until
 *    ehdg_destroy.
 *  - Pointers are HOST pointers unless the argument `on_device` is non-zero,
 *    in which case they are device pointers valid on the context's device.
 *    Device-pointer transfers are ordered on the context's stream: a call
 *    that takes device pointers may return before the stream has read them,
 *    so they must stay valid until later work on that stream (the next step,
 *    or a synchronisation of the stream) has run. Host pointers are copied
 *    before the call returns.
 *  - Meshes are conforming, axis-aligned quads (dim 2) or hexes (dim 3).
 *    Local faces are numbered f = 2*axis + side (order -x,+x,-y,+y,-z,+z).
 *    On every face the minus element sees n^- = +e_axis when it lies on the
 *    low side (interior faces) and the outward normal on boundary faces.
 *  - Volume unknowns of an element are tensor-product Lagrange values at the
 *    (p+1)^dim Gauss-Lobatto-Legendre nodes, node i = a0 + (p+1) a1 +
 *    (p+1)^2 a2; a state array is [n_elem][nf][Np] with nf = 1 (transport)
 *    or 3 (shallow water: phi, u, v).
 *  - Traces are stored by their values at the q^(dim-1) Gauss points of each
 *    face (tangential axes in increasing order, first one fastest), the
 *    points where the local equations use them: a trace array is
 *    [n_face][Nqf]. q = p+1 for a constant velocity and ceil(3p/2)+1 for a
 *    per-node velocity, which integrates every face and volume term exactly.
 */
#ifndef EHDG_H
#define EHDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ehdg_ctx_s* ehdg_ctx;

typedef enum {
  EHDG_OK = 0,
  EHDG_ERR_INVALID = 1,        /* bad argument or inconsistent mesh */
  EHDG_ERR_OOM = 2,            /* device or host memory exhausted */
  EHDG_ERR_CUDA = 3,           /* a CUDA call failed (also: no usable device or driver) */
  EHDG_ERR_NOT_CONVERGED = 4,  /* max_iter reached; state and history stay readable */
  EHDG_ERR_DIVERGED = 5,       /* non-finite residual */
  EHDG_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  EHDG_ERR_UNSUPPORTED = 7     /* size or option outside what this build supports */
} ehdg_status;

typedef enum { EHDG_TRANSPORT = 0, EHDG_SW_LINEAR = 1 } ehdg_pde;

/* Time discretisation of one implicit step. BE: backward Euler (Sec. 3).
 * CN: Crank-Nicolson, (M/dt)(u^{n+1}-u^n) + 1/2[a(u^{n+1},uhat^{n+1}) +
 * a(u^n,uhat^n)] = 1/2(F^{n+1}+F^n). STEADY: the steady problem of Sec. 3
 * (eq. transport). */
typedef enum { EHDG_BE = 0, EHDG_CN = 1, EHDG_STEADY = 2 } ehdg_scheme;

/* Precision of the element sweeps. FP64: every sweep in float64. MIXED_*:
 * defect correction on the trace fixed point -- each outer iteration is one
 * FP64 sweep (FP64 residual R = F(uhat) - uhat and the FP64 convergence test),
 * followed by `inner_sweeps` low-precision eHDG sweeps on the correction
 * equation delta = R + S H delta and the FP64 update uhat += delta; the fixed
 * point and the stopping rule are those of the FP64 iteration. MIXED_FP32 uses
 * float32 operands and accumulation on the CUDA cores.
 * FP64_EMULATED: every sweep FP64-accurate, with the element products on the
 * BF16 tensor cores by the Ozaki splitting -- each element's traces and each
 * operator row in 49-bit fixed point against their largest exponent, split
 * into seven 7-bit digits whose products are summed exactly (integers below
 * 2^24 in FP32 accumulators) and recombined in 64-bit integers; the trace
 * formula and the residual stay FP64. Per product the error is below about
 * 2^-49 (|uhat| max|Hy row| + |Hy| max|uhat_e|) + 2^-51 max|uhat_e| max|Hy row|.
 * One local operator shared by all elements (uniform mesh; transport:
 * constant velocity, 2D p <= 6 or 3D p <= 3, at most 64 sweep rows per
 * element; shallow water: no beta-plane, p <= 5), otherwise ehdg_create
 * returns EHDG_ERR_UNSUPPORTED. The step's G = P w and the reconstruction
 * u = G + H uhat run the same way where n <= 64. The paper has no
 * counterpart: it is a GB300 form of the plain FP64 path. */
typedef enum {
  EHDG_FP64 = 0,
  EHDG_MIXED_TF32 = 1,
  EHDG_MIXED_BF16 = 2,
  EHDG_MIXED_FP32 = 3,
  EHDG_FP64_EMULATED = 4
} ehdg_precision;

/* Face tags. */
enum { EHDG_FACE_INTERIOR = 0, EHDG_FACE_DIRICHLET = 1, EHDG_FACE_WALL = 2 };

/* Mesh: partition of the domain into elements K_j and the skeleton of
 * unique faces (Sec. 2). All arrays are caller-owned and copied at create. */
typedef struct {
  int dim;                     /* 2 or 3 */
  int64_t n_elem, n_face;
  const double*  elem_lo;      /* [n_elem][dim] lower corner */
  const double*  elem_h;       /* [n_elem][dim] edge lengths (> 0) */
  const int64_t* elem_face;    /* [n_elem][2*dim] face id of local face f */
  const int64_t* face_elem;    /* [n_face][2] minus, plus element; plus = -1 on the boundary */
  const int8_t*  face_local;   /* [n_face][2] local face on each side; -1 for a missing plus */
  const int32_t* face_tag;     /* [n_face] EHDG_FACE_*: transport boundaries must be DIRICHLET,
                                  shallow-water boundaries WALL */
} ehdg_mesh_desc;

/* Problem (Sec. 3): PDE, degree, velocity or mean depth, time step, tolerance. */
typedef struct {
  ehdg_pde pde;
  int p;                       /* polynomial degree, 1..6 (dim 2), 1..3 (dim 3) */
  ehdg_scheme scheme;
  double dt;                   /* time step (ignored for STEADY) */
  double tol;                  /* stop when ||uhat^{k+1}-uhat^k||_{L2(E_h)} < tol; >= 0 (0 runs
                                  max_iter iterations, reported as not converged) */
  int max_iter;                /* iteration cap per step, >= 1 */
  ehdg_precision precision;    /* one of ehdg_precision */
  const double* beta_const;    /* [dim] constant velocity, or NULL */
  const double* beta_nodes;    /* [n_elem][dim][Np] nodal velocity, or NULL (transport) */
  double Phi;                  /* shallow water: mean geopotential Phi > 0 */
  int inner_sweeps;            /* mixed precision: low-precision sweeps per outer
                                  iteration (0 = 8) */
  /* Shallow water source terms of eq. linearizedShallow (Sec. 3): Coriolis
   * parameter f = coriolis_f0 + coriolis_beta (y - coriolis_ym) and bottom
   * friction gamma = friction >= 0, in the local equations (eq.
   * localSolverDD). All zero gives the equations without them; transport
   * requires zeros. A nonzero coriolis_beta makes every element's operator
   * different (per-element operators). Wind stress tau / rho enters as
   * forcing of the velocity rows: ehdg_set_forcing with (tau_x, tau_y) /
   * (rho Phi) in the u and v fields. */
  double coriolis_f0;
  double coriolis_beta;
  double coriolis_ym;
  double friction;
  /* MIXED_* precisions: nonzero runs the outer FP64 sweeps (the FP64
   * residual R and the convergence test) as FP64_EMULATED sweeps on the BF16
   * tensor cores, under the same conditions as FP64_EMULATED (otherwise
   * ehdg_create returns EHDG_ERR_UNSUPPORTED). Zero: DFMA sweeps. Ignored by
   * FP64 and FP64_EMULATED. */
  int emulated_outer;
} ehdg_problem_desc;

/* Sizes of a created context. */
typedef struct {
  int dim, p, nf, Np, q, Nqf;  /* Np nodes per field, q Gauss points per axis, Nqf per face */
  int64_t n_elem, n_face;
  int64_t state_len;           /* n_elem * nf * Np */
  int64_t trace_len;           /* n_face * Nqf */
  int shared_operator;         /* 1 if one local operator serves every element */
  int64_t device_bytes;        /* device memory held by the context */
  int64_t sweep_rows;          /* face-point rows the element sweep computes, summed over
                                  elements (upwind/tangential points only for transport) */
  int sum_factorised;          /* 1 if the FP64 sweep and reconstruction apply the face term
                                  by 1D passes per face (hexahedra, one shared transport
                                  operator): per element 2 NQFS q + NQFS + rows NB FMAs per
                                  sweep, NB = (p+1)^3 - (p-1)^3 boundary nodes */
  int warm_start;              /* 1 if, after a step with at least one sweep, the next step
                                  starts from that step's final trace instead of forming the
                                  trace formula of u^n (Algorithm 1's initial trace): the last
                                  sweep wrote Ey u^n at every owned point, so only the inflow
                                  boundary points are recomputed from the new boundary data
                                  (backward Euler or steady transport on hexahedra with no
                                  beta.n = 0 point; backward-Euler shallow water, whose wall
                                  trace reads no boundary data). ehdg_set_state starts cold
                                  again. */
} ehdg_info;

/* Structured N0 x N1 (x N2) mesh of the box [lo, hi] with the numbering
 * above (faces axis by axis, axis 0 fastest within an axis); boundary faces
 * get `boundary_tag`. Arrays are library-owned: release with ehdg_mesh_free. */
ehdg_status ehdg_mesh_structured(int dim, const int64_t n[3], const double lo[3],
                                 const double hi[3], int32_t boundary_tag, ehdg_mesh_desc* out);
void ehdg_mesh_free(ehdg_mesh_desc* mesh);

/* Validate the mesh (indices in range, elem_face and face_elem consistent,
 * every local face on exactly one face, interior faces with the minus element
 * on the low side, boundary tags matching the PDE, positive finite sizes, and
 * conforming geometry: the two elements of an interior face meet on it, to
 * 1e-9 of the coordinates' magnitude; otherwise EHDG_ERR_INVALID before any
 * CUDA call), upload it, assemble every local operator of Sec. 3
 * (eq. transportLocal or localSolverDD plus the time term) on the GPU and
 * factor it. `cuda_stream` is a cudaStream_t (NULL: the legacy default
 * stream) on which all later work of the context is ordered. */
ehdg_status ehdg_create(const ehdg_mesh_desc* mesh, const ehdg_problem_desc* prob,
                        void* cuda_stream, ehdg_ctx* out);
/* Sizes of the context's arrays and the kernels it chose (ehdg_info above).
 * EHDG_ERR_INVALID for a NULL argument. */
ehdg_status ehdg_get_info(ehdg_ctx ctx, ehdg_info* out);
/* Waits for the context's stream, then frees every device and host array the
 * context owns. NULL is a no-op. The contexts of a batch belong to it and are
 * freed by ehdg_batch_destroy, not here. */
void ehdg_destroy(ehdg_ctx ctx);

/* Physical coordinates of the volume nodes [n_elem][Np][dim] and of the face
 * Gauss points [n_face][Nqf][dim] (from the minus element), host arrays. */
ehdg_status ehdg_node_coords(ehdg_ctx ctx, double* x);
ehdg_status ehdg_face_point_coords(ehdg_ctx ctx, double* x);

/* Set the state u^n [n_elem][nf][Np]. The trace of the state is the trace
 * formula applied to u with the current boundary data (Algorithm 1's initial
 * trace), unless `uhat` [n_face][Nqf] is given. */
ehdg_status ehdg_set_state(ehdg_ctx ctx, const double* u, const double* uhat, int on_device);
/* Forcing at the new time level, nodal values [n_elem][nf][Np] of the right-hand
 * side of u_t + beta.grad u = f (transport) or phi_t + Phi div vel = f_phi,
 * vel_t + grad phi = f_vel (shallow water); NULL sets zero. */
ehdg_status ehdg_set_forcing(ehdg_ctx ctx, const double* f, int on_device);
/* Boundary data g at the face points [n_face][Nqf] for the new time level
 * (entries of interior faces are ignored). Transport: the exterior value in
 * the trace formula, so uhat = g where beta.n^- < 0. Kept until replaced;
 * Crank-Nicolson also keeps the previous level's data. Only the rows of
 * boundary faces are read: from device memory (on_device) in stream order;
 * from pinned host memory through its device mapping, and from other host
 * memory by a copy of the whole array, before the call returns (the host
 * buffer may then be reused). */
ehdg_status ehdg_set_boundary(ehdg_ctx ctx, const double* g, int on_device);

/* One implicit step (Algorithm 1 from the warm start u^n). Writes the number of
 * iterations and the last residual; EHDG_ERR_NOT_CONVERGED if max_iter was
 * reached (the iterate is still the new state). */
ehdg_status ehdg_step(ehdg_ctx ctx, int* iters, double* final_residual);
/* n_steps implicit steps; iters_per_step [n_steps] may be NULL. Boundary data
 * and forcing stay as last set. */
ehdg_status ehdg_run(ehdg_ctx ctx, int n_steps, int* iters_per_step);
/* Exactly n_iter eHDG iterations of the current step from the warm start,
 * without the convergence test (the step is then completed as by ehdg_step). */
ehdg_status ehdg_step_fixed(ehdg_ctx ctx, int n_iter);

/* Copy the current state u^n [n_elem][nf][Np] and its trace uhat
 * [n_face][Nqf] (either pointer may be NULL to skip it) out of the context's
 * internal layout, into device memory (on_device) or host memory (through
 * the context's staging array). Ordered after the context's earlier work;
 * returns once the copies are complete. EHDG_ERR_INVALID for a NULL context,
 * EHDG_ERR_CUDA if a copy fails. */
ehdg_status ehdg_get_state(ehdg_ctx ctx, double* u, double* uhat, int on_device);

/* Checkpoint and resume. ehdg_save writes everything a later step depends on:
 * the state u^n, its trace, the previous step's trace (Crank-Nicolson), the
 * boundary data of the new and previous levels, and the forcing. The file
 * format is versioned: a header with the sizes and a hash of the mesh and
 * problem, then the arrays, then a CRC-32 of the arrays. ehdg_load restores
 * them into a context created with the same mesh and problem; a mismatch
 * (sizes, hash, CRC) returns EHDG_ERR_INVALID and leaves the context unchanged. */
ehdg_status ehdg_save(ehdg_ctx ctx, const char* path);
ehdg_status ehdg_load(ehdg_ctx ctx, const char* path);

/* Autotuner for the mixed-precision inner sweep count: runs one implicit step
 * from the current state with each candidate (restoring the state after each),
 * keeps the fastest, and reports it; the state is left as it was. */
ehdg_status ehdg_autotune_inner_sweeps(ehdg_ctx ctx, const int* candidates, int n_candidates,
                                       int* best, double* best_ms);
/* Autotuner for the FP64 path of a context that has both (FP64_EMULATED, or a
 * MIXED_* precision with emulated_outer): runs one implicit step from the
 * current state with the DFMA kernels and one with the tensor-core kernels
 * (restoring the state after each), keeps the faster, and reports both times;
 * the state is left as it was. Both paths are FP64-accurate; the tensor cores
 * pay on large shared-operator problems, the DFMA kernels on small ones (a
 * tensor-core launch has a fixed setup). A batch recaptures its graph after
 * an instance's path changed. EHDG_ERR_INVALID for a context without the
 * tensor-core path. The paper has no counterpart. */
ehdg_status ehdg_autotune_fp64_path(ehdg_ctx ctx, int* tensor_cores, double* ms_dfma,
                                    double* ms_tensor);
/* Autotuner for the tile shape of the fused FP64 transport sweep (shared
 * operator, or a per-element operator without a tiled kernel; also the outer
 * sweeps of mixed precision): each 32-element tile is worked by 32 x FT
 * threads, FT row groups. Candidates are FT values (2, 4 or 8; others are
 * skipped). Runs one implicit step from the current state per candidate
 * (restoring the state after each), keeps the fastest, and reports it with
 * its time; the state is left as it was. Every row is one thread's FMA chain
 * for any FT, so the iterates do not change, only the summation order of the
 * residual. A batch recaptures its graph after the choice changed.
 * EHDG_ERR_INVALID for a context whose FP64 sweep is another kernel (shallow
 * water, the tiled per-element sweep, the tensor-core FP64 path). */
ehdg_status ehdg_autotune_sweep_tile(ehdg_ctx ctx, const int* candidates, int n_candidates,
                                     int* best_ft, double* best_ms);
/* Residual history r_0, r_1, ... of the last step (host buffer of cap entries). */
ehdg_status ehdg_get_residual_history(ehdg_ctx ctx, double* buf, int64_t cap, int64_t* n_out);

/* Batched form: n independent problems (each its own mesh, degree, velocity,
 * precision) stepped together. Every implicit step of every instance is
 * captured into ONE CUDA graph (each step with its own device-side
 * convergence loop), so one graph launch advances all instances by one time
 * step. The graph has k independent branches ("chains"); each runs its
 * instances' steps one after the other, and the branches run concurrently.
 * Instances go to branches longest step first, each to the least-loaded
 * branch, by an estimate of their step's device time (iterations of their
 * last step times the sweep's work, plus a fixed latency per iteration). */
typedef struct ehdg_batch_s* ehdg_batch;
ehdg_status ehdg_batch_create(int n, const ehdg_mesh_desc* meshes, const ehdg_problem_desc* probs,
                              void* cuda_stream, ehdg_batch* out);
/* The context of instance i (owned by the batch): set its state, boundary
 * data and forcing, read its results, with the single-problem calls. */
ehdg_status ehdg_batch_instance(ehdg_batch b, int i, ehdg_ctx* out);
/* n_steps steps of every instance. iters [n][n_steps] (may be NULL) receives
 * each step's eHDG iterations; inst_time_s [n] (may be NULL) the device time
 * of each instance's branch, summed over the steps (%globaltimer). Returns
 * the first non-OK status of any instance. */
ehdg_status ehdg_batch_run(ehdg_batch b, int n_steps, int* iters, double* inst_time_s);
/* Branch count k of the batch's graph. k <= 0 (the default) takes the number
 * of hardware work queues the GPU runs concurrent branches on: the value of
 * CUDA_DEVICE_MAX_CONNECTIONS when the CUDA context was created (8 if unset,
 * at most 32). k >= n gives every instance its own branch. The graph is
 * recaptured at the next run. EHDG_ERR_INVALID for a NULL batch. */
ehdg_status ehdg_batch_set_chains(ehdg_batch b, int k);
/* Batched iteration loop (on by default). The instances it supports -- 2D
 * transport with one shared operator per instance (constant velocity,
 * uniform mesh), p <= 6, no face point with beta.n = 0, FP64 or TF32/BF16
 * mixed precision -- iterate together: the graph of a step holds their once-per-step kernels on the
 * branches and ONE conditional loop whose every iteration is one launch of
 * each of: the m correction sweeps, the FP64 update, and the FP64 sweep, each
 * over the tiles of every instance that has not converged yet (instance and
 * tile tables on the device; each instance keeps its own counter, residual
 * history and stopping test, Algorithm 1 of Sec. 3 per instance). The other
 * instances run their own loops on the branches, concurrently. An instance's
 * iterates are the same, bit for bit, either way. on = 0 runs every instance
 * on the branches. on = 2 is the loop's persistent form where every looped
 * instance is FP64 or has FP32 corrections and their largest stages fit the
 * ring of 65,536 work items together (about 8 million elements; else on = 1):
 * all iterations of a
 * step in ONE launch, each instance at its own pace -- the block that
 * completes a stage of an instance (its FP64 sweep, a correction sweep, the
 * FP64 update) publishes the next stage's work items to a ring in device
 * memory, and every block takes the next item of the ring; waits on the ring
 * are bounded (a wait that gives up makes the step EHDG_ERR_TIMEOUT). The
 * graph is recaptured at the next run. EHDG_ERR_INVALID for a NULL batch or
 * a mode outside 0..2. */
ehdg_status ehdg_batch_set_loop(ehdg_batch b, int on);
/* Kernel accounting of the batched loop (a diagnostic; the paper has no
 * counterpart). With profiling on (which resets the counters),
 * ehdg_batch_run drives the looped instances' steps from the host -- the
 * same kernels as the graph, each launch bracketed by CUDA events on the
 * batch's stream, the loop condition read back after every iteration -- and
 * runs every other instance's steps by its own graph; inst_time_s is then not
 * filled. ehdg_batch_kernel_stats returns the launches and summed device time
 * of one ehdg_kernel_kind of the looped instances' kernels: STEP right-hand
 * side, FACE initial trace and trace hand-over, ELEM FP64 sweeps, CORR
 * correction sweeps, FINAL reconstruction, AUX reset, work lists, FP64
 * update and step record. EHDG_ERR_INVALID for a NULL batch or a bad kind. */
ehdg_status ehdg_batch_set_profiling(ehdg_batch b, int on);
ehdg_status ehdg_batch_kernel_stats(ehdg_batch b, int kind, int64_t* launches, double* total_ms);
/* Autotuner for the branch count: from the instances' current states, each
 * candidate k runs as many batch steps as the batch's last ehdg_batch_run
 * (one step before the first run) -- the run the choice is for -- timed with
 * CUDA events on the batch's stream, every instance's state restored after
 * each; keeps the fastest candidate and reports it with its time (of all
 * those steps). The states are left as they were. EHDG_ERR_INVALID for a
 * NULL batch or no candidates. */
ehdg_status ehdg_batch_autotune_chains(ehdg_batch b, const int* candidates, int n_candidates,
                                       int* best, double* best_ms);
/* Autotuner for the schedule of a batch step (the paper has no counterpart):
 * times the batched loop (every instance it supports iterates in one loop of
 * launches over the unconverged instances), its persistent form
 * (ehdg_batch_set_loop mode 2) and every instance's own loop on k graph
 * branches, k from chain_candidates (entries < 1 skipped), and keeps the
 * fastest. Same protocol as ehdg_batch_autotune_chains (each candidate timed
 * over the batch's last run, states restored). *loop_on (may be NULL)
 * receives the kept ehdg_batch_set_loop mode (0 branches, 1 loop, 2
 * persistent), *chains the branch count kept, *best_ms the time of the kept
 * schedule. Every schedule gives the same iterates bit for bit.
 * EHDG_ERR_INVALID for a NULL batch or no candidates. */
ehdg_status ehdg_batch_autotune_schedule(ehdg_batch b, const int* chain_candidates,
                                         int n_candidates, int* loop_on, int* chains,
                                         double* best_ms);
/* Autotuner for the tile shape (FT, as in ehdg_autotune_sweep_tile) of every
 * instance's fused FP64 sweep together, timed as whole batch steps: instances
 * that share the GPU favour other shapes than one instance alone. Same
 * protocol as ehdg_batch_autotune_chains; instances whose sweep is another
 * kernel are unaffected. EHDG_ERR_INVALID for a NULL batch or no candidates. */
ehdg_status ehdg_batch_autotune_sweep_tile(ehdg_batch b, const int* candidates, int n_candidates,
                                           int* best_ft, double* best_ms);
/* Autotuner for the inner sweep count m (1..64; others are skipped) of every
 * mixed-precision instance together, timed as whole batch steps; same
 * protocol as ehdg_batch_autotune_chains. FP64 instances are unaffected.
 * EHDG_ERR_INVALID for a NULL batch, no candidates, or a batch without a
 * mixed-precision instance. */
ehdg_status ehdg_batch_autotune_inner_sweeps(ehdg_batch b, const int* candidates,
                                             int n_candidates, int* best_m, double* best_ms);
/* Waits for the batch's stream, then destroys its graph, its streams, its
 * device arrays and every instance's context (the handles ehdg_batch_instance
 * returned become invalid). NULL is a no-op. */
void ehdg_batch_destroy(ehdg_batch b);

/* FP64 residual of Algorithm 1's convergence check (Sec. 3, "check
 * convergence"): out[0] = sqrt(sum_i w[i] (a[i] - b[i])^2) over n entries.
 * With a, b two trace iterates uhat^{k+1}, uhat^k at the face points and w the
 * face Gauss weights times the face Jacobian, this is
 * ||uhat^{k+1} - uhat^k||_{L2(E_h)}. All pointers are device pointers; the
 * work is ordered on `stream` (a cudaStream_t, NULL = legacy default). The
 * reduction is deterministic (same inputs give the same bits). Scratch for
 * the block partial sums is allocated on the stream and released before the
 * call returns. n = 0 gives 0 (a, b and w may then be NULL); n < 0, a NULL
 * out, or a NULL data pointer with n > 0 is EHDG_ERR_INVALID. */
ehdg_status ehdg_trace_residual(const double* a, const double* b, const double* w, int64_t n,
                                double* out, void* stream);

/* Allocation-free variant of ehdg_trace_residual. The paper has no
 * counterpart: this exists for callers that cannot allocate device memory,
 * such as code running under a host application's memory manager that owns
 * every device allocation, or code in latency-critical loops where
 * cudaMalloc/cudaFree would synchronise the device. It computes the same
 * out[0] = sqrt(sum_i w[i] (a[i] - b[i])^2) with the same kernel, but the block
 * partial sums live in a fixed device array inside the library (8 KB plus a
 * ticket word, 256-byte aligned), which every GPU that loads the library holds
 * until the process exits. It calls no cudaMalloc, cudaFree or other
 * allocating routine. n may be at most EHDG_NOALLOC_MAX_N, a fixed limit of this
 * entry point (the array itself does not depend on n); larger n returns
 * EHDG_ERR_UNSUPPORTED with a message. The first call on a device looks up the
 * array's device address (once per device, with that device current) and
 * keeps it for the life of the process, so make that first call before any
 * stream capture; a cudaDeviceReset between calls is not supported. All calls share the one array:
 * calls that overlap on the GPU (different streams, or concurrent host threads
 * on one device) race and may return wrong results; order them on one stream. */
#define EHDG_NOALLOC_MAX_N 16777216LL
ehdg_status ehdg_trace_residual_noalloc(const double* a, const double* b, const double* w,
                                        int64_t n, double* out, void* stream);

/* Self-test of the bounded device-side waits (the paper has no
 * counterpart). which = 0 runs the mbarrier waits of the tiled sweeps,
 * which = 1 the grid barrier of the persistent sweep, which = 2 the work-ring
 * wait of the persistent batched loop. Each runs against a condition that
 * never holds: an mbarrier that no arrival completes, a barrier target one
 * arrival beyond the grid, or a ring with a live instance where nothing is
 * ever published. The poll limit is short, so
 * the call takes milliseconds. Every wait must give up and report it through a
 * flag the host reads. The expected result is EHDG_ERR_TIMEOUT; EHDG_OK means a
 * wait did not give up, which is a defect. The device stays usable afterwards.
 * stream: a cudaStream_t or NULL; the call synchronises it. */
ehdg_status ehdg_selftest_wait_timeout(int which, void* stream);

/* Measured FP64 FMA rate of the current device (a diagnostic; the paper has no
 * counterpart). Runs a kernel in which every thread carries 8 independent
 * fma() chains, 4 blocks of 256 threads per SM, 2^14 steps per chain, on
 * `stream` (a cudaStream_t or NULL), once to warm up and three times timed
 * with CUDA events; *tflops receives 2 flops x FMAs / the fastest time in
 * TFLOP/s, *sms (may be NULL) the SM count it ran on. It is the measured
 * denominator of the FP64 sweeps' roofline. Synchronises the stream; allocates
 * nothing. EHDG_ERR_INVALID for a NULL tflops, EHDG_ERR_CUDA if a launch or
 * event call fails. */
ehdg_status ehdg_probe_fp64_rate(void* stream, int* sms, double* tflops);

/* Kernel accounting. Every launch is counted per kind; with profiling on,
 * each launch is also bracketed by CUDA events on the context's stream and
 * ehdg_kernel_stats returns the summed device time of the kind (it
 * synchronises the stream). With profiling on, ehdg_step and ehdg_run drive
 * the iteration from the host (one launch per kernel, the same kernels and
 * iterates as the graph) so that every launch can be timed. ehdg_set_profiling
 * (either value) synchronises the stream and resets the counters. */
typedef enum {
  EHDG_KERNEL_ASSEMBLE = 0,    /* local operator assembly + factorisation (setup) */
  EHDG_KERNEL_SIGNS = 1,       /* sgn(beta.n) at face points (setup) */
  EHDG_KERNEL_STEP = 2,        /* per-step right-hand side G = P w */
  EHDG_KERNEL_ELEM = 3,        /* element sweep Y = Gy + Hy uhat */
  EHDG_KERNEL_FACE = 4,        /* trace formula + residual */
  EHDG_KERNEL_FINAL = 5,       /* end-of-step reconstruction */
  EHDG_KERNEL_AUX = 6,         /* transposes, extraction, resets, the mixed FP64 update */
  EHDG_KERNEL_CORR = 7,        /* low-precision correction sweeps of mixed precision */
  EHDG_KERNEL_KINDS = 8
} ehdg_kernel_kind;
ehdg_status ehdg_set_profiling(ehdg_ctx ctx, int on);
ehdg_status ehdg_kernel_stats(ehdg_ctx ctx, int kind, int64_t* launches, double* total_ms);

/* Message of the last failed call on the calling thread (the message is
 * kept per thread; a later failure replaces it). The pointer stays valid until
 * the thread's next failing call. */
const char* ehdg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EHDG_H */
