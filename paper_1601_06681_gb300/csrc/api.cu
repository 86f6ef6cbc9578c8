// C ABI of libehdg: validation, device memory, per-step orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ehdg_internal.h"

using namespace ehdg;


struct ehdg_batch_s {
  std::vector<ehdg_ctx> inst;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> branch;
  cudaStream_t cap = nullptr, body = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<char> graph_force;
  std::vector<int> graph_gen;          // each instance's path_gen when the graph was captured
  unsigned long long* t_start = nullptr;
  unsigned long long* t_acc = nullptr;
  int chains = 0;                       // concurrent branches of the graph (<= 0: automatic)
  bool built_on_estimate = false;       // the graph's schedule used estimated iteration counts
  // batched iteration loop (one launch per kernel and iteration over every
  // unconverged instance) for the instances it supports
  bool use_loop = true;
  // its persistent form (every iteration of a step in one launch), where the
  // looped instances allow it (FP64 or FP32 corrections)
  bool use_persist = false;
  int last_run_steps = 0;               // steps of the last run: what the autotuners time
  // kernel accounting of the batched loop (ehdg_batch_set_profiling)
  bool profiling = false;
  double prof_ms[EHDG_KERNEL_KINDS] = {0};
  int64_t prof_launches[EHDG_KERNEL_KINDS] = {0};
  bool tuning = false;                  // an autotuner is running candidate steps
  ehdg::BatchLoop loop;
  std::vector<char> looped;             // instance i iterates in the batched loop
  unsigned long long* t_conv = nullptr; // convergence time of each instance in a step
};

namespace {

thread_local std::string g_err;

ehdg_status fail(ehdg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

ehdg_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return EHDG_ERR_CUDA;
}

#define CK(expr)                                          \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);   \
  } while (0)

template <class T>
ehdg_status dalloc(Ctx& c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    // out of memory is EHDG_ERR_OOM; any other failure (no device, no
    // driver, a sticky error) is a CUDA error
    return fail(e == cudaErrorMemoryAllocation ? EHDG_ERR_OOM : EHDG_ERR_CUDA,
                std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  c.allocs.push_back(q);
  c.bytes += (int64_t)(count * sizeof(T));
  *p = static_cast<T*>(q);
  return EHDG_OK;
}

#define TRY(expr)                         \
  do {                                    \
    ehdg_status _s = (expr);              \
    if (_s != EHDG_OK) return _s;         \
  } while (0)

int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

ehdg_status validate_mesh(const ehdg_mesh_desc* m, ehdg_pde pde) {
  if (!m) return fail(EHDG_ERR_INVALID, "mesh is NULL");
  if (m->dim != 2 && m->dim != 3) return fail(EHDG_ERR_INVALID, "dim must be 2 or 3");
  if (m->n_elem < 1 || m->n_face < 1) return fail(EHDG_ERR_INVALID, "empty mesh");
  if (m->n_elem >= (1LL << 31) || m->n_face >= (1LL << 31))
    return fail(EHDG_ERR_UNSUPPORTED, "more than 2^31-1 elements or faces");
  if (!m->elem_lo || !m->elem_h || !m->elem_face || !m->face_elem || !m->face_local || !m->face_tag)
    return fail(EHDG_ERR_INVALID, "mesh array is NULL");
  const int dim = m->dim, F = 2 * dim;
  for (int64_t e = 0; e < m->n_elem * dim; ++e)
    if (!(m->elem_h[e] > 0.0) || !std::isfinite(m->elem_h[e]) || !std::isfinite(m->elem_lo[e]))
      return fail(EHDG_ERR_INVALID, "element sizes must be positive and finite");
  std::vector<int> seen((size_t)m->n_elem * F, 0);
  for (int64_t f = 0; f < m->n_face; ++f) {
    const int64_t em = m->face_elem[2 * f], ep = m->face_elem[2 * f + 1];
    const int lm = m->face_local[2 * f], lp = m->face_local[2 * f + 1];
    if (em < 0 || em >= m->n_elem || ep < -1 || ep >= m->n_elem || lm < 0 || lm >= F)
      return fail(EHDG_ERR_INVALID, "face " + std::to_string(f) + ": bad element or local face");
    if (m->elem_face[em * F + lm] != f)
      return fail(EHDG_ERR_INVALID, "face " + std::to_string(f) + ": elem_face/face_elem mismatch");
    seen[em * F + lm]++;
    const int tag = m->face_tag[f];
    if (ep >= 0) {
      if (lp < 0 || lp >= F || m->elem_face[ep * F + lp] != f)
        return fail(EHDG_ERR_INVALID, "face " + std::to_string(f) + ": bad plus side");
      if ((lm & 1) != 1 || lp != lm - 1)
        return fail(EHDG_ERR_INVALID, "face " + std::to_string(f) +
                                          ": interior faces need the minus element on the low side");
      if (tag != EHDG_FACE_INTERIOR)
        return fail(EHDG_ERR_INVALID, "interior face with a boundary tag");
      // conforming geometry: along the face's normal axis the plus element
      // starts where the minus element ends, and along every other axis the
      // two span the same interval (to rounding, relative to the coordinates)
      const int ax = lm >> 1;
      const double* lo_m = m->elem_lo + em * dim;
      const double* h_m = m->elem_h + em * dim;
      const double* lo_p = m->elem_lo + ep * dim;
      const double* h_p = m->elem_h + ep * dim;
      for (int a = 0; a < dim; ++a) {
        const double scale = std::max(std::fabs(lo_m[a]) + h_m[a], std::fabs(lo_p[a]) + h_p[a]);
        const double off = (a == ax) ? lo_m[a] + h_m[a] - lo_p[a] : lo_m[a] - lo_p[a];
        const double dh = (a == ax) ? 0.0 : h_m[a] - h_p[a];
        if (std::fabs(off) > 1e-9 * scale || std::fabs(dh) > 1e-9 * scale)
          return fail(EHDG_ERR_INVALID, "face " + std::to_string(f) +
                                            ": the elements on its two sides do not meet on it "
                                            "(non-conforming mesh)");
      }
      seen[ep * F + lp]++;
    } else {
      if (lp != -1) return fail(EHDG_ERR_INVALID, "boundary face with a plus local face");
      const int want = (pde == EHDG_TRANSPORT) ? EHDG_FACE_DIRICHLET : EHDG_FACE_WALL;
      if (tag != want)
        return fail(EHDG_ERR_INVALID, pde == EHDG_TRANSPORT
                                          ? "transport boundary faces must be tagged DIRICHLET"
                                          : "shallow-water boundary faces must be tagged WALL");
    }
  }
  for (size_t i = 0; i < seen.size(); ++i)
    if (seen[i] != 1) return fail(EHDG_ERR_INVALID, "every local face must belong to exactly one face");
  return EHDG_OK;
}

cudaEvent_t pool_event(Ctx& c) {
  if (!c.ev_pool.empty()) {
    cudaEvent_t e = c.ev_pool.back();
    c.ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch through `fn`, counting `n` kernels of `kind`; with profiling on the
// launch is bracketed by events on the context's stream.
template <class Fn>
cudaError_t counted(Ctx& c, int kind, int n, Fn fn) {
  c.launches[kind] += n;
  if (!c.profiling) return fn();
  cudaEvent_t a = pool_event(c), b = pool_event(c);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, c.stream);
  if (e != cudaSuccess) return e;
  e = fn();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(b, c.stream);
  if (e != cudaSuccess) return e;
  c.ev_used.push_back({kind, a, b});
  return cudaSuccess;
}

ehdg_status upload(Ctx& c, double* dst_soa, const double* src, int64_t outer, int inner,
                   int on_device) {
  const double* s = src;
  if (!on_device) {
    CK(cudaMemcpyAsync(c.staging, src, sizeof(double) * outer * inner, cudaMemcpyHostToDevice,
                       c.stream));
    s = c.staging;
  }
  CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_aos_to_soa(s, dst_soa, outer, inner, c.stream); }));
  if (!on_device) CK(cudaStreamSynchronize(c.stream));
  return EHDG_OK;
}

ehdg_status download(Ctx& c, double* dst, const double* src_soa, int64_t outer, int inner,
                     int on_device) {
  double* d = on_device ? dst : c.staging;
  CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_soa_to_aos(src_soa, d, outer, inner, c.stream); }));
  if (!on_device) {
    CK(cudaMemcpyAsync(dst, c.staging, sizeof(double) * outer * inner, cudaMemcpyDeviceToHost,
                       c.stream));
    CK(cudaStreamSynchronize(c.stream));
  }
  return EHDG_OK;
}

// Kernels of one step right-hand side: the tensor-core G = P w, if used,
// before the step kernel.
int step_launches(const Ctx& c) { return (c.use_ozaki && c.oz_step.img) ? 2 : 1; }

// A tensor-core sweep whose bounded mbarrier wait gave up leaves a flag.
ehdg_status check_tc_err(Ctx& c) {
  if (!c.tc_err) return EHDG_OK;
  int te = 0;
  CK(cudaMemcpy(&te, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (te) return fail(EHDG_ERR_TIMEOUT, "a sweep's bounded mbarrier wait gave up");
  return EHDG_OK;
}

ehdg_status run_step(Ctx& c, int fixed_iters, int* iters, double* res) {
  CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_reset_iter(c); }));
  CK(counted(c, EHDG_KERNEL_STEP, step_launches(c), [&] { return launch_step(c); }));
  CK(counted(c, EHDG_KERNEL_FACE, face_launches(c, kFaceInitial),
             [&] { return launch_face(c, kFaceInitial); }));
  const int n_it = fixed_iters > 0 ? fixed_iters : c.max_iter;
  bool persist = fixed_iters <= 0 && persistent_sweep_ok(c);
  if (persist) {   // every iteration of the step in one cooperative launch
    if (counted(c, EHDG_KERNEL_ELEM, 1, [&] { return launch_sweep_persistent(c); }) !=
        cudaSuccess) {
      // not launchable here (e.g. the grid cannot be co-resident): iterate
      // with one launch per sweep from now on
      cudaGetLastError();
      c.launches[EHDG_KERNEL_ELEM] -= 1;
      c.persist_fits = false;
      persist = false;
    }
  }
  for (int k = 0; k < (persist ? 0 : n_it); ++k) {
    if (k > 0 && c.mixed) {
      // low-precision correction of uhat before the next FP64 sweep: m inner
      // sweeps (each timed on its own with profiling on), then the FP64 update
      const float* in = c.R32;
      const bool fuse = tc_apply_fusable(c);   // the last inner sweep makes the FP64 update
      for (int j = 0; j < c.inner_sweeps; ++j) {
        float* out = correction_out(c, j);
        const bool last = fuse && j == c.inner_sweeps - 1;
        CK(counted(c, EHDG_KERNEL_CORR, lp_sweep_launches(c),
                   [&] { return launch_lp_sweep(c, in, out, last); }));
        in = out;
      }
      if (!fuse) CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_apply(c, in); }));
    }
    if (c.pde == EHDG_TRANSPORT) {
      // element solve + trace formula + residual in one kernel (+ tangential points)
      CK(counted(c, EHDG_KERNEL_ELEM, 1, [&] { return launch_sweep_fused(c, 0); }));
      if (c.n_tan > 0) c.launches[EHDG_KERNEL_FACE] += 1;
    } else {
      CK(counted(c, EHDG_KERNEL_ELEM, 1, [&] { return launch_elem(c); }));
      CK(counted(c, EHDG_KERNEL_FACE, 1, [&] { return launch_face(c, kFaceIterate); }));
    }
    if (fixed_iters <= 0) {
      CK(cudaMemcpyAsync(c.it_host, c.it, sizeof(IterState), cudaMemcpyDeviceToHost, c.stream));
      CK(cudaStreamSynchronize(c.stream));
      if (!c.it_host->cont) break;
    }
  }
  CK(counted(c, EHDG_KERNEL_FINAL, 2, [&] { return launch_final(c); }));
  if (c.have_force)
    CK(cudaMemcpyAsync(c.force_old, c.force, sizeof(double) * c.n * c.nel,
                       cudaMemcpyDeviceToDevice, c.stream));
  CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_step_end(c); }));
  CK(cudaMemcpyAsync(c.it_host, c.it, sizeof(IterState), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  c.last_iters = std::min(c.it_host->k, c.max_iter);
  if (iters) *iters = c.it_host->k;
  if (res) *res = c.it_host->r_last;
  TRY(check_tc_err(c));
  if (fixed_iters > 0) return EHDG_OK;
  const ehdg_status st = (ehdg_status)c.it_host->status;
  if (st == EHDG_ERR_NOT_CONVERGED) return fail(st, "eHDG did not reach the tolerance in max_iter iterations");
  if (st == EHDG_ERR_DIVERGED) return fail(st, "non-finite eHDG residual");
  return st;
}

void destroy_graph(Ctx& c) {
  if (c.gexec) cudaGraphExecDestroy(c.gexec);
  if (c.graph) cudaGraphDestroy(c.graph);
  c.gexec = nullptr;
  c.graph = nullptr;
}

// End-of-step kernels of a captured step: reconstruction, forcing copy,
// bookkeeping.
ehdg_status capture_step_end(Ctx& c) {
  cudaError_t err;
  if ((err = launch_final(c)) != cudaSuccess) return cuda_fail(err, "capture final");
  if (c.have_force &&
      (err = cudaMemcpyAsync(c.force_old, c.force, sizeof(double) * c.n * c.nel,
                             cudaMemcpyDeviceToDevice, c.stream)) != cudaSuccess)
    return cuda_fail(err, "capture forcing copy");
  if ((err = launch_step_end(c)) != cudaSuccess) return cuda_fail(err, "capture step end");
  return EHDG_OK;
}

// Append one implicit step of context c to the graph being captured on
// stream s: reset, step RHS, initial trace, then a WHILE node whose body is
// {element sweep, trace update} (mixed precision: an FP64 sweep before the
// loop and {correction, FP64 sweep} as the body); the sweep's last block sets
// the condition (continue while r_k >= tol and k < max_iter), so the
// iteration runs without a host round trip; then the end-of-step kernels.
// body_stream is a spare stream used to capture the loop body.
ehdg_status capture_step(Ctx& c, cudaStream_t s, cudaStream_t body_stream, bool allow_persist) {
  cudaStream_t user = c.stream;
  struct Restore {
    Ctx& c;
    cudaStream_t s;
    ~Restore() { c.stream = s; }
  } restore{c, user};
  c.stream = s;
  cudaError_t err = cudaSuccess;
  if ((err = launch_reset_iter(c)) != cudaSuccess) return cuda_fail(err, "capture reset");
  if ((err = launch_step(c)) != cudaSuccess) return cuda_fail(err, "capture step");
  if ((err = launch_face(c, kFaceInitial)) != cudaSuccess) return cuda_fail(err, "capture face");
  if (allow_persist && persistent_sweep_ok(c)) {
    // every iteration in one cooperative launch: no conditional node needed
    if ((err = launch_sweep_persistent(c)) != cudaSuccess)
      return cuda_fail(err, "capture persistent sweep");
    c.graph_persist = true;
    return capture_step_end(c);
  }
  c.graph_persist = false;
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle handle;
  err = cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, nullptr, nullptr, nullptr);
  if (err != cudaSuccess) return cuda_fail(err, "cudaStreamGetCaptureInfo");
  err = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGraphConditionalHandleCreate");
  c.handle = handle;
  if (c.mixed) {
    err = (c.pde == EHDG_TRANSPORT) ? launch_sweep_fused(c, 1) : launch_elem(c);
    if (err == cudaSuccess && c.pde != EHDG_TRANSPORT) err = launch_face(c, kFaceIterate, 1);
    if (err != cudaSuccess) return cuda_fail(err, "capture first FP64 sweep");
  }
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  err = cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps);
  if (err != cudaSuccess) return cuda_fail(err, "cudaStreamGetCaptureInfo");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cond;
  err = cudaGraphAddNode(&cond, g, deps, nullptr, ndeps, &cp);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGraphAddNode(while)");
  err = cudaStreamUpdateCaptureDependencies(s, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (err != cudaSuccess) return cuda_fail(err, "cudaStreamUpdateCaptureDependencies");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  err = cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  if (err != cudaSuccess) return cuda_fail(err, "cudaStreamBeginCaptureToGraph");
  c.stream = body_stream;
  cudaError_t e2 = cudaSuccess;
  if (c.mixed) e2 = launch_correction(c);
  if (e2 == cudaSuccess) {
    if (c.pde == EHDG_TRANSPORT) {
      e2 = launch_sweep_fused(c, 1);
    } else {
      e2 = launch_elem(c);
      if (e2 == cudaSuccess) e2 = launch_face(c, kFaceIterate, 1);
    }
  }
  cudaError_t e3 = cudaStreamEndCapture(body_stream, &body);
  c.stream = s;
  if (e2 != cudaSuccess) return cuda_fail(e2, "capture loop body");
  if (e3 != cudaSuccess) return cuda_fail(e3, "end body capture");
  return capture_step_end(c);
}

void abort_capture(cudaStream_t s) {
  cudaGraph_t junk = nullptr;
  cudaStreamEndCapture(s, &junk);
  if (junk) cudaGraphDestroy(junk);
  cudaGetLastError();
}

ehdg_status try_build_graph(Ctx& c, bool allow_persist) {
  destroy_graph(c);
  if (!c.cap_stream) CK(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  if (!c.body_stream) CK(cudaStreamCreateWithFlags(&c.body_stream, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeRelaxed));
  const ehdg_status st = capture_step(c, c.cap_stream, c.body_stream, allow_persist);
  if (st != EHDG_OK) {
    const std::string msg = g_err;
    abort_capture(c.cap_stream);
    g_err = msg;
    return st;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamEndCapture(c.cap_stream, &g));
  c.graph = g;
  CK(cudaGraphInstantiate(&c.gexec, g, 0));
  c.graph_force = c.have_force;
  return EHDG_OK;
}

// The step graph; a step whose persistent sweep cannot be captured or
// instantiated falls back to the conditional loop of per-iteration sweeps.
ehdg_status build_graph(Ctx& c) {
  const bool want = persistent_sweep_ok(c);
  ehdg_status st = try_build_graph(c, want);
  if (st != EHDG_OK && want) {
    cudaGetLastError();
    c.persist_fits = false;
    st = try_build_graph(c, false);
  }
  return st;
}

ehdg_status ensure_step_arrays(Ctx& c, int n) {
  if (n <= c.step_cap) return EHDG_OK;
  int cap = std::max(n, 64);
  int *a = nullptr, *b = nullptr;
  TRY(dalloc(c, &a, cap));
  TRY(dalloc(c, &b, cap));
  c.step_iters = a;
  c.step_status = b;
  c.step_cap = cap;
  destroy_graph(c);   // the graph holds the old pointers
  return EHDG_OK;
}

// n_steps implicit steps as back-to-back graph launches; one sync at the end.
ehdg_status run_graph(Ctx& c, int n_steps, int* iters_per_step, double* res) {
  TRY(ensure_step_arrays(c, n_steps));
  if (!c.gexec || c.graph_force != c.have_force) TRY(build_graph(c));
  CK(cudaMemsetAsync(&c.it->step, 0, sizeof(int), c.stream));
  for (int s = 0; s < n_steps; ++s) CK(cudaGraphLaunch(c.gexec, c.stream));
  c.launches[EHDG_KERNEL_AUX] += 2 * n_steps;   // reset + step end
  c.launches[EHDG_KERNEL_STEP] += (int64_t)n_steps * step_launches(c);
  c.launches[EHDG_KERNEL_FINAL] += 2 * n_steps;
  c.step_iters_h.resize(n_steps);
  c.step_status_h.resize(n_steps);
  CK(cudaMemcpyAsync(c.step_iters_h.data(), c.step_iters, sizeof(int) * n_steps,
                     cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(c.step_status_h.data(), c.step_status, sizeof(int) * n_steps,
                     cudaMemcpyDeviceToHost, c.stream));
  CK(cudaMemcpyAsync(c.it_host, c.it, sizeof(IterState), cudaMemcpyDeviceToHost, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  ehdg_status first = EHDG_OK;
  int64_t sweeps = 0;
  for (int s = 0; s < n_steps; ++s) {
    sweeps += c.step_iters_h[s];
    if (iters_per_step) iters_per_step[s] = c.step_iters_h[s];
    if (first == EHDG_OK && c.step_status_h[s] != EHDG_OK) first = (ehdg_status)c.step_status_h[s];
  }
  c.launches[EHDG_KERNEL_ELEM] += c.graph_persist ? n_steps : sweeps;
  c.launches[EHDG_KERNEL_FACE] += (int64_t)n_steps * face_launches(c, kFaceInitial) +
                                   ((c.pde == EHDG_TRANSPORT) ? (c.n_tan > 0 ? sweeps : 0) : sweeps);
  if (c.mixed) {
    c.launches[EHDG_KERNEL_CORR] += (sweeps - n_steps) * c.inner_sweeps * lp_sweep_launches(c);
    // the FP64 update: its own launch unless the last inner sweep makes it
    if (!tc_apply_fusable(c)) c.launches[EHDG_KERNEL_AUX] += sweeps - n_steps;
  }
  c.last_iters = n_steps > 0 ? std::min(c.step_iters_h[n_steps - 1], c.max_iter) : 0;
  if (res) *res = c.it_host->r_last;
  TRY(check_tc_err(c));
  if (first == EHDG_ERR_NOT_CONVERGED) return fail(first, "eHDG did not reach the tolerance in max_iter iterations");
  if (first == EHDG_ERR_DIVERGED) return fail(first, "non-finite eHDG residual");
  return first;
}

}  // namespace

namespace ehdg {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace ehdg

extern "C" {

const char* ehdg_last_error(void) { return g_err.c_str(); }

ehdg_status ehdg_set_profiling(ehdg_ctx h, int on) {
  if (!h) return fail(EHDG_ERR_INVALID, "NULL context");
  Ctx& c = h->c;
  CK(cudaStreamSynchronize(c.stream));
  for (auto& r : c.ev_used) {
    c.ev_pool.push_back(r.a);
    c.ev_pool.push_back(r.b);
  }
  c.ev_used.clear();
  for (int k = 0; k < EHDG_KERNEL_KINDS; ++k) c.launches[k] = 0;
  c.profiling = on != 0;
  return EHDG_OK;
}

ehdg_status ehdg_kernel_stats(ehdg_ctx h, int kind, int64_t* launches, double* total_ms) {
  if (!h || kind < 0 || kind >= EHDG_KERNEL_KINDS) return fail(EHDG_ERR_INVALID, "bad argument");
  Ctx& c = h->c;
  CK(cudaStreamSynchronize(c.stream));
  double ms = 0.0;
  for (auto& r : c.ev_used) {
    if (r.kind != kind) continue;
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
  }
  if (launches) *launches = c.launches[kind];
  if (total_ms) *total_ms = ms;
  return EHDG_OK;
}

ehdg_status ehdg_mesh_structured(int dim, const int64_t n[3], const double lo[3], const double hi[3],
                                 int32_t boundary_tag, ehdg_mesh_desc* out) {
  if (!out || !n || !lo || !hi) return fail(EHDG_ERR_INVALID, "NULL argument");
  if (dim != 2 && dim != 3) return fail(EHDG_ERR_INVALID, "dim must be 2 or 3");
  int64_t N[3] = {1, 1, 1};
  int64_t nel = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 1) return fail(EHDG_ERR_INVALID, "mesh size must be >= 1");
    if (!(hi[a] > lo[a])) return fail(EHDG_ERR_INVALID, "hi must exceed lo");
    N[a] = n[a];
    nel *= n[a];
  }
  int64_t nface = 0;
  for (int ax = 0; ax < dim; ++ax) {
    int64_t c = 1;
    for (int a = 0; a < dim; ++a) c *= (a == ax) ? N[a] + 1 : N[a];
    nface += c;
  }
  const int F = 2 * dim;
  double* elo = (double*)std::malloc(sizeof(double) * nel * dim);
  double* eh = (double*)std::malloc(sizeof(double) * nel * dim);
  int64_t* ef = (int64_t*)std::malloc(sizeof(int64_t) * nel * F);
  int64_t* fe = (int64_t*)std::malloc(sizeof(int64_t) * nface * 2);
  int8_t* fl = (int8_t*)std::malloc(sizeof(int8_t) * nface * 2);
  int32_t* ft = (int32_t*)std::malloc(sizeof(int32_t) * nface);
  if (!elo || !eh || !ef || !fe || !fl || !ft) {
    std::free(elo); std::free(eh); std::free(ef); std::free(fe); std::free(fl); std::free(ft);
    return fail(EHDG_ERR_OOM, "host allocation failed");
  }
  const int64_t stride[3] = {1, N[0], N[0] * N[1]};
  for (int64_t e = 0; e < nel; ++e) {
    int64_t rem = e;
    for (int a = 0; a < dim; ++a) {
      const int64_t i = rem % N[a];
      rem /= N[a];
      const double h = (hi[a] - lo[a]) / (double)N[a];
      elo[e * dim + a] = lo[a] + (double)i * h;
      eh[e * dim + a] = h;
    }
  }
  int64_t fid = 0;
  for (int ax = 0; ax < dim; ++ax) {
    int64_t shape[3];
    int64_t cnt = 1;
    for (int a = 0; a < dim; ++a) {
      shape[a] = (a == ax) ? N[a] + 1 : N[a];
      cnt *= shape[a];
    }
    for (int64_t col = 0; col < cnt; ++col, ++fid) {
      int64_t ii[3] = {0, 0, 0}, rem = col;
      for (int a = 0; a < dim; ++a) {
        ii[a] = rem % shape[a];
        rem /= shape[a];
      }
      const int64_t k = ii[ax];
      int64_t base = 0;
      for (int a = 0; a < dim; ++a) base += (a == ax ? 0 : ii[a]) * stride[a];
      if (k > 0 && k < N[ax]) {
        const int64_t em = base + (k - 1) * stride[ax], ep = base + k * stride[ax];
        fe[2 * fid] = em; fe[2 * fid + 1] = ep;
        fl[2 * fid] = (int8_t)(2 * ax + 1); fl[2 * fid + 1] = (int8_t)(2 * ax);
        ft[fid] = EHDG_FACE_INTERIOR;
        ef[em * F + 2 * ax + 1] = fid;
        ef[ep * F + 2 * ax] = fid;
      } else if (k == 0) {
        const int64_t em = base;
        fe[2 * fid] = em; fe[2 * fid + 1] = -1;
        fl[2 * fid] = (int8_t)(2 * ax); fl[2 * fid + 1] = -1;
        ft[fid] = boundary_tag;
        ef[em * F + 2 * ax] = fid;
      } else {
        const int64_t em = base + (k - 1) * stride[ax];
        fe[2 * fid] = em; fe[2 * fid + 1] = -1;
        fl[2 * fid] = (int8_t)(2 * ax + 1); fl[2 * fid + 1] = -1;
        ft[fid] = boundary_tag;
        ef[em * F + 2 * ax + 1] = fid;
      }
    }
  }
  out->dim = dim;
  out->n_elem = nel;
  out->n_face = nface;
  out->elem_lo = elo;
  out->elem_h = eh;
  out->elem_face = ef;
  out->face_elem = fe;
  out->face_local = fl;
  out->face_tag = ft;
  return EHDG_OK;
}

void ehdg_mesh_free(ehdg_mesh_desc* m) {
  if (!m) return;
  std::free((void*)m->elem_lo);
  std::free((void*)m->elem_h);
  std::free((void*)m->elem_face);
  std::free((void*)m->face_elem);
  std::free((void*)m->face_local);
  std::free((void*)m->face_tag);
  std::memset(m, 0, sizeof(*m));
}

static void release(Ctx& c) {
  destroy_graph(c);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  if (c.body_stream) cudaStreamDestroy(c.body_stream);
  c.cap_stream = c.body_stream = nullptr;
  for (auto& r : c.ev_used) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c.ev_pool) cudaEventDestroy(e);
  c.ev_used.clear();
  c.ev_pool.clear();
  for (void* p : c.allocs) cudaFree(p);
  c.allocs.clear();
  if (c.it_host) cudaFreeHost(c.it_host);
  c.it_host = nullptr;
}

ehdg_status ehdg_create(const ehdg_mesh_desc* mesh, const ehdg_problem_desc* prob, void* stream,
                        ehdg_ctx* out) {
  if (!out) return fail(EHDG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!prob) return fail(EHDG_ERR_INVALID, "problem is NULL");
  if (prob->pde != EHDG_TRANSPORT && prob->pde != EHDG_SW_LINEAR)
    return fail(EHDG_ERR_INVALID, "unknown pde");
  TRY(validate_mesh(mesh, prob->pde));
  const int dim = mesh->dim, p = prob->p;
  if (prob->precision != EHDG_FP64 && prob->precision != EHDG_MIXED_FP32 &&
      prob->precision != EHDG_MIXED_TF32 && prob->precision != EHDG_MIXED_BF16 &&
      prob->precision != EHDG_FP64_EMULATED)
    return fail(EHDG_ERR_INVALID, "unknown precision");
  if (prob->inner_sweeps < 0 || prob->inner_sweeps > 64)
    return fail(EHDG_ERR_INVALID, "inner_sweeps must be 0..64");
  if (prob->scheme != EHDG_BE && prob->scheme != EHDG_CN && prob->scheme != EHDG_STEADY)
    return fail(EHDG_ERR_INVALID, "unknown scheme");
  if (prob->scheme != EHDG_STEADY && !(prob->dt > 0.0 && std::isfinite(prob->dt)))
    return fail(EHDG_ERR_INVALID, "dt must be positive");
  if (!(prob->tol >= 0.0) || prob->max_iter < 1) return fail(EHDG_ERR_INVALID, "bad tol or max_iter");
  if (p < 1 || (dim == 2 && p > 6) || (dim == 3 && p > 3))
    return fail(EHDG_ERR_UNSUPPORTED, "p must be 1..6 in 2D and 1..3 in 3D");
  bool variable = false;
  if (prob->pde == EHDG_TRANSPORT) {
    if ((prob->beta_const == nullptr) == (prob->beta_nodes == nullptr))
      return fail(EHDG_ERR_INVALID, "give exactly one of beta_const and beta_nodes");
    variable = prob->beta_nodes != nullptr;
  } else {
    if (dim != 2) return fail(EHDG_ERR_UNSUPPORTED, "shallow water is 2D");
    if (!(prob->Phi > 0.0)) return fail(EHDG_ERR_INVALID, "Phi must be positive");
    if (p > 5) return fail(EHDG_ERR_UNSUPPORTED, "shallow water supports p <= 5");
  }
  const double src_terms[4] = {prob->coriolis_f0, prob->coriolis_beta, prob->coriolis_ym,
                               prob->friction};
  for (double v : src_terms)
    if (!std::isfinite(v)) return fail(EHDG_ERR_INVALID, "Coriolis and friction must be finite");
  if (prob->friction < 0.0) return fail(EHDG_ERR_INVALID, "friction must be >= 0");
  if (prob->pde == EHDG_TRANSPORT && (prob->coriolis_f0 != 0.0 || prob->coriolis_beta != 0.0 ||
                                      prob->friction != 0.0))
    return fail(EHDG_ERR_INVALID, "Coriolis and friction are shallow-water terms");
  const int q = variable ? (3 * p + 1) / 2 + 1 : p + 1;
  if (q > kMaxQ || p + 1 > kMaxP1) return fail(EHDG_ERR_UNSUPPORTED, "degree too high");

  ehdg_ctx h = new (std::nothrow) ehdg_ctx_s();
  if (!h) return fail(EHDG_ERR_OOM, "host allocation failed");
  Ctx& c = h->c;
  c.dim = dim;
  c.p = p;
  c.pde = prob->pde;
  c.scheme = prob->scheme;
  c.nf = prob->pde == EHDG_TRANSPORT ? 1 : 3;
  c.Np = ipow(p + 1, dim);
  c.n = c.nf * c.Np;
  c.q = q;
  c.Nqf = ipow(q, dim - 1);
  c.F = 2 * dim;
  c.NQFS = c.F * c.Nqf;
  c.nel = mesh->n_elem;
  c.nface = mesh->n_face;
  c.dt = prob->dt;
  // Crank-Nicolson runs as its midpoint form: a backward-Euler stage of dt/2
  // for v = (u^n + u^{n+1})/2, then u^{n+1} = 2 v - u^n (same iterates).
  c.dt_eff = prob->scheme == EHDG_CN ? 0.5 * prob->dt : prob->dt;
  c.res_scale = prob->scheme == EHDG_CN ? 2.0 : 1.0;
  c.tol = prob->tol;
  c.max_iter = prob->max_iter;
  c.Phi = prob->Phi;
  c.cor_f0 = prob->coriolis_f0;
  c.cor_beta = prob->coriolis_beta;
  c.cor_ym = prob->coriolis_ym;
  c.friction = prob->friction;
  c.variable_beta = variable;
  c.mixed = prob->precision != EHDG_FP64 && prob->precision != EHDG_FP64_EMULATED;
  c.precision = prob->precision;
  c.inner_sweeps = prob->inner_sweeps > 0 ? prob->inner_sweeps : 8;
  c.stream = (cudaStream_t)stream;
  if (prob->pde == EHDG_TRANSPORT && !variable)
    for (int a = 0; a < dim; ++a) c.beta_const[a] = prob->beta_const[a];

  bool uniform = true;
  for (int64_t e = 1; e < c.nel && uniform; ++e)
    for (int a = 0; a < dim; ++a)
      if (mesh->elem_h[e * dim + a] != mesh->elem_h[a]) uniform = false;
  // a beta-plane Coriolis parameter varies with y: one operator per element
  c.shared_op = uniform && !variable && !(prob->pde == EHDG_SW_LINEAR && c.cor_beta != 0.0);
  if (c.precision == EHDG_MIXED_TF32 && !c.shared_op) {
    delete h;
    return fail(EHDG_ERR_UNSUPPORTED,
                "TF32 tensor-core sweeps need one local operator shared by all elements "
                "(constant velocity, uniform mesh); use EHDG_MIXED_FP32 or EHDG_MIXED_BF16");
  }
  const bool want_ozaki =
      c.precision == EHDG_FP64_EMULATED || (c.mixed && prob->emulated_outer != 0);
  if (want_ozaki && !c.shared_op) {
    delete h;
    return fail(EHDG_ERR_UNSUPPORTED,
                "FP64_EMULATED sweeps need one local operator shared by all elements (uniform "
                "mesh; transport: constant velocity; shallow water: no beta-plane)");
  }
  if (c.precision == EHDG_MIXED_BF16 && !c.shared_op && prob->pde != EHDG_TRANSPORT) {
    delete h;
    return fail(EHDG_ERR_UNSUPPORTED,
                "BF16 correction sweeps with per-element operators are built for transport");
  }

  build_ref1d(p, q, &c.r1d);
  c.ref.dim = dim;
  c.ref.p = p;
  c.ref.q = q;
  c.ref.Np = c.Np;
  c.ref.Nqf = c.Nqf;
  c.ref.nf = c.nf;
  for (int g = 0; g < q; ++g) {
    c.ref.om[g] = c.r1d.om[g];
    c.ref.xi[g] = c.r1d.xi[g];
    for (int a = 0; a <= p; ++a) {
      c.ref.L[g * kMaxP1 + a] = c.r1d.L[g * (p + 1) + a];
      c.ref.D[g * kMaxP1 + a] = c.r1d.D[g * (p + 1) + a];
    }
  }
  for (int s = 0; s < 2; ++s)
    for (int a = 0; a <= p; ++a) c.ref.Lend[s * kMaxP1 + a] = c.r1d.Lend[s * (p + 1) + a];

  // face-point extraction Ey: element values at the face points
  // (transport: u; shallow water: c = (phi + sqrt(Phi) vel.n_f) / 2)
  std::vector<std::vector<std::pair<int, double>>> ey(c.NQFS);
  const int n1 = p + 1;
  for (int f = 0; f < c.F; ++f) {
    const int ax = f >> 1, side = f & 1;
    for (int gf = 0; gf < c.Nqf; ++gf) {
      for (int i = 0; i < c.Np; ++i) {
        int rem = i, t = 0, gr = gf;
        double v = 1.0;
        for (int a = 0; a < dim; ++a) {
          const int ia = rem % n1;
          rem /= n1;
          if (a == ax) {
            v *= c.r1d.Lend[side * n1 + ia];
          } else {
            const int ga = gr % q;
            gr /= q;
            v *= c.r1d.L[ga * n1 + ia];
            ++t;
          }
        }
        if (v == 0.0) continue;
        const int s = f * c.Nqf + gf;
        if (c.pde == EHDG_TRANSPORT) {
          ey[s].push_back({i, v});
        } else {
          ey[s].push_back({i, 0.5 * v});
          ey[s].push_back({(1 + ax) * c.Np + i, 0.5 * std::sqrt(c.Phi) * (side ? 1.0 : -1.0) * v});
        }
      }
    }
  }
  c.KE = 0;
  for (auto& r : ey) c.KE = std::max<int>(c.KE, (int)r.size());
  std::vector<int> eyi((size_t)c.NQFS * c.KE, 0);
  std::vector<double> eyv((size_t)c.NQFS * c.KE, 0.0);
  for (int s = 0; s < c.NQFS; ++s)
    for (size_t k = 0; k < ey[s].size(); ++k) {
      eyi[s * c.KE + k] = ey[s][k].first;
      eyv[s * c.KE + k] = ey[s][k].second;
    }
  // rows each element must produce: for a constant velocity only the faces
  // where it is upwind (first) or tangential (eq. transportLocale reads those)
  std::vector<int> rows;
  int n_up = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int s = 0; s < c.NQFS; ++s) {
      const int f = s / c.Nqf, ax = f >> 1;
      if (c.pde == EHDG_TRANSPORT && !variable) {
        const double bn = ((f & 1) ? 1.0 : -1.0) * c.beta_const[ax];
        if (pass == 0 ? !(bn > 0.0) : !(bn == 0.0)) continue;
      } else if (pass == 1) {
        continue;
      }
      rows.push_back(s);
    }
    if (pass == 0) n_up = (int)rows.size();
  }
  c.n_up = n_up;
  c.n_rows = (int)rows.size();
  c.rows_host = rows;

  // shared memory needed by the assembly kernel
  {
    int Q = ipow(q, dim);
    size_t smem = sizeof(double) * ((size_t)c.n * (2 * c.n + c.NQFS) + dim * c.Np + 2 * dim * Q +
                                    c.F * c.Nqf + c.n);
    if (smem > 220 * 1024) {
      delete h;
      return fail(EHDG_ERR_UNSUPPORTED, "local system too large for on-chip assembly");
    }
  }

  // host copies
  c.elem_lo.assign(mesh->elem_lo, mesh->elem_lo + c.nel * dim);
  c.elem_h.assign(mesh->elem_h, mesh->elem_h + c.nel * dim);
  c.face_elem_h.assign(mesh->face_elem, mesh->face_elem + 2 * c.nface);
  c.face_local_h.assign(mesh->face_local, mesh->face_local + 2 * c.nface);
  c.elem_face_h.assign(mesh->elem_face, mesh->elem_face + c.F * c.nel);

  auto cleanup = [&](ehdg_status s) {
    std::string msg = g_err;
    release(c);
    delete h;
    g_err = msg;
    return s;
  };
#define TRYC(expr)                               \
  do {                                           \
    ehdg_status _s = (expr);                     \
    if (_s != EHDG_OK) return cleanup(_s);       \
  } while (0)
#define CKC(expr)                                                      \
  do {                                                                 \
    cudaError_t _e = (expr);                                           \
    if (_e != cudaSuccess) return cleanup(cuda_fail(_e, #expr));       \
  } while (0)

  // geometry in SoA / int32
  std::vector<int32_t> ef32((size_t)c.F * c.nel), fe32((size_t)2 * c.nface);
  std::vector<int8_t> fl8((size_t)2 * c.nface), tag8(c.nface);
  std::vector<double> jf(c.nface);
  for (int64_t e = 0; e < c.nel; ++e)
    for (int f = 0; f < c.F; ++f) ef32[f * c.nel + e] = (int32_t)mesh->elem_face[e * c.F + f];
  for (int64_t f = 0; f < c.nface; ++f) {
    fe32[f] = (int32_t)mesh->face_elem[2 * f];
    fe32[c.nface + f] = (int32_t)mesh->face_elem[2 * f + 1];
    fl8[f] = mesh->face_local[2 * f];
    fl8[c.nface + f] = mesh->face_local[2 * f + 1];
    tag8[f] = (int8_t)mesh->face_tag[f];
    const int64_t em = mesh->face_elem[2 * f];
    const int ax = mesh->face_local[2 * f] >> 1;
    double v = 1.0;
    for (int a = 0; a < dim; ++a)
      if (a != ax) v *= 0.5 * mesh->elem_h[em * dim + a];
    jf[f] = v;
  }
  double* d_h = nullptr;
  int32_t *d_ef = nullptr, *d_fe = nullptr;
  int8_t *d_fl = nullptr, *d_tag = nullptr;
  double* d_jf = nullptr;
  TRYC(dalloc(c, &d_h, (size_t)c.nel * dim));
  TRYC(dalloc(c, &d_ef, ef32.size()));
  TRYC(dalloc(c, &d_fe, fe32.size()));
  TRYC(dalloc(c, &d_fl, fl8.size()));
  TRYC(dalloc(c, &d_tag, tag8.size()));
  TRYC(dalloc(c, &d_jf, jf.size()));
  CKC(cudaMemcpy(d_h, mesh->elem_h, sizeof(double) * c.nel * dim, cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(d_ef, ef32.data(), sizeof(int32_t) * ef32.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(d_fe, fe32.data(), sizeof(int32_t) * fe32.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(d_fl, fl8.data(), fl8.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(d_tag, tag8.data(), tag8.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(d_jf, jf.data(), sizeof(double) * jf.size(), cudaMemcpyHostToDevice));
  c.geo.nel = c.nel;
  c.geo.nface = c.nface;
  c.geo.elem_h = d_h;
  c.geo.elem_face = d_ef;
  c.geo.face_elem = d_fe;
  c.geo.face_local = d_fl;
  c.geo.face_tag = d_tag;
  c.geo.face_jf = d_jf;
  {
    // boundary faces: the only ones whose boundary data the steps read
    std::vector<int32_t> bf;
    for (int64_t f = 0; f < c.nface; ++f)
      if (c.face_elem_h[2 * f + 1] < 0) bf.push_back((int32_t)f);
    c.n_bface = (int64_t)bf.size();
    if (!bf.empty()) {
      TRYC(dalloc(c, &c.bface, bf.size()));
      CKC(cudaMemcpy(c.bface, bf.data(), sizeof(int32_t) * bf.size(), cudaMemcpyHostToDevice));
    }
  }

  const int64_t ne = c.shared_op ? 1 : c.nel;
  TRYC(dalloc(c, &c.P, (size_t)c.n * c.n * ne));
  TRYC(dalloc(c, &c.H, (size_t)c.n * c.NQFS * ne));
  TRYC(dalloc(c, &c.Hy, (size_t)c.NQFS * c.NQFS * ne));
  TRYC(dalloc(c, &c.ey_idx, eyi.size()));
  TRYC(dalloc(c, &c.ey_val, eyv.size()));
  TRYC(dalloc(c, &c.rows, rows.size()));
  CKC(cudaMemcpy(c.ey_idx, eyi.data(), sizeof(int) * eyi.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(c.ey_val, eyv.data(), sizeof(double) * eyv.size(), cudaMemcpyHostToDevice));
  CKC(cudaMemcpy(c.rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice));
  if (c.pde == EHDG_SW_LINEAR && (c.cor_f0 != 0.0 || c.cor_beta != 0.0)) {
    TRYC(dalloc(c, &c.elem_lo_d, (size_t)c.nel * dim));
    CKC(cudaMemcpy(c.elem_lo_d, c.elem_lo.data(), sizeof(double) * c.nel * dim,
                   cudaMemcpyHostToDevice));
  }
  if (variable) {
    TRYC(dalloc(c, &c.beta_nodes, (size_t)c.nel * dim * c.Np));
    CKC(cudaMemcpy(c.beta_nodes, prob->beta_nodes, sizeof(double) * c.nel * dim * c.Np,
                   cudaMemcpyHostToDevice));
    // checkpoints identify the velocity field by this hash (FNV-1a of the bytes)
    uint64_t hb = 1469598103934665603ull;
    const unsigned char* bp = reinterpret_cast<const unsigned char*>(prob->beta_nodes);
    for (size_t i = 0; i < sizeof(double) * (size_t)c.nel * dim * c.Np; ++i) {
      hb ^= bp[i];
      hb *= 1099511628211ull;
    }
    c.beta_nodes_hash = hb;
  }
  const size_t state = (size_t)c.n * c.nel, trace = (size_t)c.Nqf * c.nface;
  TRYC(dalloc(c, &c.sgn, trace));
  if (!c.shared_op) {
    if (c.NQFS > 255) return cleanup(fail(EHDG_ERR_UNSUPPORTED, "more than 255 face points per element"));
    TRYC(dalloc(c, &c.rowid, (size_t)c.NQFS * c.nel));
    TRYC(dalloc(c, &c.nrows, (size_t)c.nel));
    TRYC(dalloc(c, &c.nup, (size_t)c.nel));
  }
  TRYC(dalloc(c, &c.u, state));
  TRYC(dalloc(c, &c.G, state));
  TRYC(dalloc(c, &c.Gy, (size_t)c.NQFS * c.nel));
  TRYC(dalloc(c, &c.Y, (size_t)c.NQFS * c.nel));
  TRYC(dalloc(c, &c.uhat, 2 * trace));
  TRYC(dalloc(c, &c.uhat_n, trace));
  TRYC(dalloc(c, &c.gb, trace));
  TRYC(dalloc(c, &c.gb_old, trace));
  TRYC(dalloc(c, &c.force, state));
  TRYC(dalloc(c, &c.force_old, state));
  TRYC(dalloc(c, &c.staging, std::max(state, trace)));
  c.n_partials = std::max(face_grid_x(c.nface, c.Nqf) * c.Nqf,
                          fused_grid(c.nel) + tangent_grid((int64_t)trace));
  TRYC(dalloc(c, &c.partials, (size_t)c.n_partials));
  if (c.mixed) {
    TRYC(dalloc(c, &c.Hy32, (size_t)c.NQFS * c.NQFS * ne));
    TRYC(dalloc(c, &c.R32, trace));
    TRYC(dalloc(c, &c.d32, 2 * trace));
    TRYC(dalloc(c, &c.Y32, (size_t)c.NQFS * c.nel));
    // points no sweep owns (inflow boundary) keep R = delta = 0 for good
    CKC(cudaMemsetAsync(c.R32, 0, sizeof(float) * trace, c.stream));
    CKC(cudaMemsetAsync(c.d32, 0, sizeof(float) * 2 * trace, c.stream));
    CKC(cudaMemsetAsync(c.Y32, 0, sizeof(float) * c.NQFS * c.nel, c.stream));
  }
  TRYC(dalloc(c, &c.tc_err, 1));
  CKC(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
  TRYC(dalloc(c, &c.it, 1));
  TRYC(dalloc(c, &c.warm, 1));
  CKC(cudaMemsetAsync(c.warm, 0, sizeof(int), c.stream));
  TRYC(dalloc(c, &c.hist, (size_t)c.max_iter));
  CKC(cudaMallocHost(&c.it_host, sizeof(IterState)));
  CKC(cudaMemsetAsync(c.u, 0, sizeof(double) * state, c.stream));
  CKC(cudaMemsetAsync(c.Y, 0, sizeof(double) * c.NQFS * c.nel, c.stream));
  CKC(cudaMemsetAsync(c.uhat, 0, sizeof(double) * 2 * trace, c.stream));
  CKC(cudaMemsetAsync(c.uhat_n, 0, sizeof(double) * trace, c.stream));
  CKC(cudaMemsetAsync(c.gb, 0, sizeof(double) * trace, c.stream));
  CKC(cudaMemsetAsync(c.gb_old, 0, sizeof(double) * trace, c.stream));
  CKC(cudaMemsetAsync(c.hist, 0, sizeof(double) * c.max_iter, c.stream));

  CKC(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_reset_iter(c); }));
  if (sf_supported(c)) {
    // sum-factorised sweep and reconstruction: the assembly also returns the
    // boundary-node columns of A^{-1} (if its shared memory still fits)
    TRYC(sf_prepare(c));
    if (asm_smem(c) <= 220 * 1024) {
      c.use_sf = true;
    } else {
      c.sf_Dy = nullptr;
      c.sf_Ab = nullptr;
    }
  }
  CKC(counted(c, EHDG_KERNEL_ASSEMBLE, 1, [&] { return launch_assemble(c, c.shared_op ? 1 : (int)c.nel); }));
  if (c.pde == EHDG_TRANSPORT)
    CKC(counted(c, EHDG_KERNEL_SIGNS, 1, [&] { return launch_face_signs(c); }));
  if (!c.shared_op) CKC(counted(c, EHDG_KERNEL_AUX, 2, [&] { return launch_rows(c); }));
  if (tiled_supported(c)) CKC(counted(c, EHDG_KERNEL_AUX, 1, [&] { return build_tiled_operator(c); }));
  if (c.precision == EHDG_MIXED_BF16 && !c.shared_op && !c.Hyt16)
    return cleanup(fail(EHDG_ERR_UNSUPPORTED,
                        "BF16 correction sweeps with per-element operators need a face-point "
                        "count of the tiled sweep (quadrilaterals with 2..10 points per edge, "
                        "hexahedra with 2x2 or 3x3 per face)"));
  if (c.mixed) CKC(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_hy_to_f32(c); }));
  if (c.mixed) CKC(counted(c, EHDG_KERNEL_AUX, 1, [&] { return build_tc_image(c); }));
  if (want_ozaki) {
    if (!ozaki_supported(c))
      return cleanup(fail(EHDG_ERR_UNSUPPORTED,
                          "FP64_EMULATED sweeps support at most 64 sweep rows and 96 face "
                          "points per element (shallow water: 24)"));
    CKC(counted(c, EHDG_KERNEL_AUX, 1, [&] { return build_ozaki_operator(c); }));
    c.use_ozaki = true;
  }
  CKC(cudaMemcpyAsync(c.it_host, c.it, sizeof(IterState), cudaMemcpyDeviceToHost, c.stream));
  CKC(cudaStreamSynchronize(c.stream));
  if (c.it_host->status != 0) return cleanup(fail(EHDG_ERR_INVALID, "singular local operator"));
  if (c.pde == EHDG_TRANSPORT) {
    // face points with beta.n = 0 (average of both sides), finished after the sweep
    std::vector<int8_t> sg((size_t)trace);
    CKC(cudaMemcpy(sg.data(), c.sgn, trace, cudaMemcpyDeviceToHost));
    std::vector<int32_t> tg, tf;
    for (int g = 0; g < c.Nqf; ++g)
      for (int64_t f = 0; f < c.nface; ++f)
        if (sg[(size_t)g * c.nface + f] == 0) {
          tg.push_back(g);
          tf.push_back((int32_t)f);
        }
    c.n_tan = (int64_t)tg.size();
    // 2D contexts keep the cold start, so that the batched loop's once-per-step
    // kernels (2D only) and solo runs stay equal bit for bit
    c.warm_ok = c.dim == 3 && c.scheme != EHDG_CN && c.n_tan == 0;
    if (c.n_tan > 0) {
      TRYC(dalloc(c, &c.tan_g, tg.size()));
      TRYC(dalloc(c, &c.tan_face, tf.size()));
      CKC(cudaMemcpy(c.tan_g, tg.data(), sizeof(int32_t) * tg.size(), cudaMemcpyHostToDevice));
      CKC(cudaMemcpy(c.tan_face, tf.data(), sizeof(int32_t) * tf.size(), cudaMemcpyHostToDevice));
    }
  }
  if (c.pde == EHDG_SW_LINEAR) {
    // shallow water: the trace formula reads no boundary data (walls), so a
    // warm step starts from the previous step's final trace unchanged (no
    // shallow-water instance iterates in the batched loop)
    c.warm_ok = c.scheme != EHDG_CN;
  }
  if (pe_supported(c)) {
    // one thread per element for the 2D shared-operator FP64 sweep
    std::vector<double> fw(kMaxQ * kMaxQ, 0.0);
    fill_face_weights(c, fw.data());
    TRYC(dalloc(c, &c.pe_fw, (size_t)c.Nqf));
    CKC(cudaMemcpy(c.pe_fw, fw.data(), sizeof(double) * c.Nqf, cudaMemcpyHostToDevice));
    if (c.n_partials < (c.nel + 127) / 128) {
      TRYC(dalloc(c, &c.partials, (size_t)((c.nel + 127) / 128)));
      c.n_partials = (int)((c.nel + 127) / 128);
    }
    c.use_pe = true;
  }
  if (c.shared_op) {
    c.sweep_rows = (int64_t)c.n_rows * c.nel;
  } else {
    std::vector<uint8_t> nr(c.nel);
    CKC(cudaMemcpy(nr.data(), c.nrows, c.nel, cudaMemcpyDeviceToHost));
    c.sweep_rows = 0;
    for (uint8_t v : nr) c.sweep_rows += v;
  }
  *out = h;
  return EHDG_OK;
}

ehdg_status ehdg_get_info(ehdg_ctx h, ehdg_info* out) {
  if (!h || !out) return fail(EHDG_ERR_INVALID, "NULL argument");
  const Ctx& c = h->c;
  out->dim = c.dim;
  out->p = c.p;
  out->nf = c.nf;
  out->Np = c.Np;
  out->q = c.q;
  out->Nqf = c.Nqf;
  out->n_elem = c.nel;
  out->n_face = c.nface;
  out->state_len = (int64_t)c.n * c.nel;
  out->trace_len = (int64_t)c.Nqf * c.nface;
  out->shared_operator = c.shared_op ? 1 : 0;
  out->device_bytes = c.bytes;
  out->sweep_rows = c.sweep_rows;
  out->sum_factorised = c.use_sf ? 1 : 0;
  out->warm_start = c.warm_ok ? 1 : 0;
  return EHDG_OK;
}

void ehdg_destroy(ehdg_ctx h) {
  if (!h) return;
  cudaStreamSynchronize(h->c.stream);
  release(h->c);
  delete h;
}

ehdg_status ehdg_node_coords(ehdg_ctx h, double* x) {
  if (!h || !x) return fail(EHDG_ERR_INVALID, "NULL argument");
  const Ctx& c = h->c;
  const int n1 = c.p + 1;
  for (int64_t e = 0; e < c.nel; ++e)
    for (int i = 0; i < c.Np; ++i) {
      int rem = i;
      for (int a = 0; a < c.dim; ++a) {
        const int ia = rem % n1;
        rem /= n1;
        x[(e * c.Np + i) * c.dim + a] =
            c.elem_lo[e * c.dim + a] + c.elem_h[e * c.dim + a] * (c.r1d.r[ia] + 1.0) / 2.0;
      }
    }
  return EHDG_OK;
}

ehdg_status ehdg_face_point_coords(ehdg_ctx h, double* x) {
  if (!h || !x) return fail(EHDG_ERR_INVALID, "NULL argument");
  const Ctx& c = h->c;
  for (int64_t f = 0; f < c.nface; ++f) {
    const int64_t em = c.face_elem_h[2 * f];
    const int lf = c.face_local_h[2 * f], ax = lf >> 1, side = lf & 1;
    for (int g = 0; g < c.Nqf; ++g) {
      int rem = g;
      for (int a = 0; a < c.dim; ++a) {
        double r;
        if (a == ax) {
          r = side ? 1.0 : -1.0;
        } else {
          r = c.r1d.xi[rem % c.q];
          rem /= c.q;
        }
        x[(f * c.Nqf + g) * c.dim + a] =
            c.elem_lo[em * c.dim + a] + c.elem_h[em * c.dim + a] * (r + 1.0) / 2.0;
      }
    }
  }
  return EHDG_OK;
}

ehdg_status ehdg_set_state(ehdg_ctx h, const double* u, const double* uhat, int on_device) {
  if (!h || !u) return fail(EHDG_ERR_INVALID, "NULL argument");
  Ctx& c = h->c;
  const size_t trace = (size_t)c.Nqf * c.nface;
  TRY(upload(c, c.u, u, c.nel, c.n, on_device));
  // a new state: the next step forms its initial trace from u (cold start)
  CK(cudaMemsetAsync(c.warm, 0, sizeof(int), c.stream));
  // the state's own level: boundary data of this level on both sides of CN's average
  CK(cudaMemcpyAsync(c.gb_old, c.gb, sizeof(double) * trace, cudaMemcpyDeviceToDevice, c.stream));
  if (uhat) {
    TRY(upload(c, c.uhat, uhat, c.nface, c.Nqf, on_device));
  } else {
    CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_extract(c); }));
    CK(counted(c, EHDG_KERNEL_FACE, face_launches(c, kFaceInitial),
               [&] { return launch_face(c, kFaceInitial); }));
  }
  CK(cudaMemcpyAsync(c.uhat_n, c.uhat, sizeof(double) * trace, cudaMemcpyDeviceToDevice, c.stream));
  // device pointers are ordered on the context's stream like every later
  // call: nothing to wait for (host pointers were copied synchronously)
  return EHDG_OK;
}

ehdg_status ehdg_set_forcing(ehdg_ctx h, const double* f, int on_device) {
  if (!h) return fail(EHDG_ERR_INVALID, "NULL context");
  Ctx& c = h->c;
  if (!f) {
    c.have_force = false;
    return EHDG_OK;
  }
  TRY(upload(c, c.force, f, c.nel, c.n, on_device));
  if (!c.have_force)
    CK(cudaMemcpyAsync(c.force_old, c.force, sizeof(double) * c.n * c.nel,
                       cudaMemcpyDeviceToDevice, c.stream));
  CK(cudaStreamSynchronize(c.stream));
  c.have_force = true;
  return EHDG_OK;
}

ehdg_status ehdg_set_boundary(ehdg_ctx h, const double* g, int on_device) {
  if (!h || !g) return fail(EHDG_ERR_INVALID, "NULL argument");
  Ctx& c = h->c;
  // only boundary faces' values are read: from device memory directly, from
  // pinned host memory through its device mapping (then the host buffer is
  // free again when the call returns); other host memory is copied whole
  const double* src = on_device ? g : nullptr;
  if (!on_device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, g) == cudaSuccess && a.type == cudaMemoryTypeHost &&
        a.devicePointer != nullptr)
      src = static_cast<const double*>(a.devicePointer);
    else
      cudaGetLastError();
  }
  if (!src) return upload(c, c.gb, g, c.nface, c.Nqf, on_device);
  CK(counted(c, EHDG_KERNEL_AUX, 1, [&] { return launch_gather_boundary(c, src, c.gb); }));
  if (!on_device) CK(cudaStreamSynchronize(c.stream));
  return EHDG_OK;
}

ehdg_status ehdg_step(ehdg_ctx h, int* iters, double* final_residual) {
  if (!h) return fail(EHDG_ERR_INVALID, "NULL context");
  // with profiling on, the host-driven loop brackets every kernel with events
  if (h->c.profiling) return run_step(h->c, 0, iters, final_residual);
  return run_graph(h->c, 1, iters, final_residual);
}

ehdg_status ehdg_run(ehdg_ctx h, int n_steps, int* iters_per_step) {
  if (!h || n_steps < 0) return fail(EHDG_ERR_INVALID, "bad argument");
  if (n_steps == 0) return EHDG_OK;
  if (!h->c.profiling) return run_graph(h->c, n_steps, iters_per_step, nullptr);
  for (int s = 0; s < n_steps; ++s) {
    int it = 0;
    const ehdg_status st = run_step(h->c, 0, &it, nullptr);
    if (iters_per_step) iters_per_step[s] = it;
    if (st != EHDG_OK) return st;
  }
  return EHDG_OK;
}

ehdg_status ehdg_step_fixed(ehdg_ctx h, int n_iter) {
  if (!h || n_iter < 1) return fail(EHDG_ERR_INVALID, "bad argument");
  return run_step(h->c, n_iter, nullptr, nullptr);
}

ehdg_status ehdg_get_state(ehdg_ctx h, double* u, double* uhat, int on_device) {
  if (!h) return fail(EHDG_ERR_INVALID, "NULL context");
  Ctx& c = h->c;
  if (u) TRY(download(c, u, c.u, c.nel, c.n, on_device));
  if (uhat) TRY(download(c, uhat, c.uhat, c.nface, c.Nqf, on_device));
  CK(cudaStreamSynchronize(c.stream));
  return EHDG_OK;
}

ehdg_status ehdg_get_residual_history(ehdg_ctx h, double* buf, int64_t cap, int64_t* n_out) {
  if (!h || (!buf && cap > 0)) return fail(EHDG_ERR_INVALID, "bad argument");
  Ctx& c = h->c;
  const int64_t n = std::min<int64_t>(c.last_iters, cap);
  if (n > 0) {
    CK(cudaMemcpyAsync(buf, c.hist, sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
  }
  if (n_out) *n_out = c.last_iters;
  return EHDG_OK;
}


static void batch_destroy_graph(ehdg_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Hardware work queues the GPU runs concurrent branches on: the value of
// CUDA_DEVICE_MAX_CONNECTIONS the CUDA driver read at context creation (8 if
// unset, at most 32).
static int hw_queues() {
  const char* v = std::getenv("CUDA_DEVICE_MAX_CONNECTIONS");
  const int q = v ? std::atoi(v) : 8;
  return std::min(32, std::max(1, q > 0 ? q : 8));
}

// Estimated device seconds of one implicit step of context c: per iteration a
// fixed latency (launches of the loop body) plus the sweep's FP64 products at
// an effective rate; the iteration count of the last step, or a guess from
// the mesh diameter before the first.
static double step_cost(const Ctx& c, bool* estimated) {
  const bool guess = c.last_iters <= 0;
  if (guess) *estimated = true;
  const double iters = guess ? std::pow((double)c.nel, 1.0 / c.dim) + 10.0 : (double)c.last_iters;
  const double rows = c.sweep_rows > 0 ? (double)c.sweep_rows : (double)c.NQFS * c.nel;
  const double m = c.mixed ? (double)c.inner_sweeps : 0.0;
  const double per_iter = 5e-6 * (1.0 + m) + 2.0 * rows * c.NQFS * (1.0 + 0.3 * m) / 5e11;
  return iters * per_iter;
}

// Instances of each branch: longest-processing-time-first onto k branches
// (each next-largest step to the least-loaded branch).
static std::vector<std::vector<int>> batch_schedule(ehdg_batch b, int k, bool* estimated) {
  const int n = (int)b->inst.size();
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) cost[i] = step_cost(b->inst[i]->c, estimated);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<std::vector<int>> lists(k);
  std::vector<double> load(k, 0.0);
  for (int i : order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lists[j].push_back(i);
    load[j] += cost[i];
  }
  return lists;
}

// One graph: fork from a start event into k branch streams, capture the
// steps of each branch's instances there one after the other (each stamped
// with %globaltimer), join back.
static ehdg_status batch_build_graph_branches(ehdg_batch b) {
  batch_destroy_graph(b);
  const int n = (int)b->inst.size();
  const int k = std::min(n, b->chains > 0 ? b->chains : hw_queues());
  bool estimated = false;
  const std::vector<std::vector<int>> lists = batch_schedule(b, k, &estimated);
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(k, nullptr);
  CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (int j = 0; j < k; ++j) CK(cudaEventCreateWithFlags(&joins[j], cudaEventDisableTiming));
  auto cleanup_events = [&]() {
    cudaEventDestroy(fork);
    for (auto e : joins) cudaEventDestroy(e);
  };
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cleanup_events();
    return cuda_fail(e, "batch capture");
  }
  e = cudaEventRecord(fork, b->cap);
  int started = 0;                                // branches forked so far
  for (int j = 0; j < k && e == cudaSuccess; ++j) {
    cudaStream_t s = b->branch[j];
    e = cudaStreamWaitEvent(s, fork, 0);
    if (e != cudaSuccess) break;
    started = j + 1;
    for (int i : lists[j]) {
      Ctx& c = b->inst[i]->c;
      if ((e = launch_stamp(s, b->t_start, b->t_acc, i, 0)) != cudaSuccess) break;
      const ehdg_status st = capture_step(c, s, b->body, false);
      if (st != EHDG_OK) {
        const std::string msg = g_err;
        for (int jj = 0; jj < started; ++jj) {
          cudaEventRecord(joins[jj], b->branch[jj]);
          cudaStreamWaitEvent(b->cap, joins[jj], 0);
        }
        abort_capture(b->cap);
        cleanup_events();
        g_err = msg;
        return st;
      }
      if ((e = launch_stamp(s, b->t_start, b->t_acc, i, 1)) != cudaSuccess) break;
      b->graph_force[i] = c.have_force ? 1 : 0;
      b->graph_gen[i] = c.path_gen;
    }
    if (e == cudaSuccess) e = cudaEventRecord(joins[j], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, joins[j], 0);
  }
  if (e != cudaSuccess) {
    for (int jj = 0; jj < started; ++jj) {
      cudaEventRecord(joins[jj], b->branch[jj]);
      cudaStreamWaitEvent(b->cap, joins[jj], 0);
    }
    abort_capture(b->cap);
    cleanup_events();
    return cuda_fail(e, "batch capture");
  }
  b->built_on_estimate = estimated;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap, &g);
  cleanup_events();
  if (e != cudaSuccess) return cuda_fail(e, "batch end capture");
  b->graph = g;
  CK(cudaGraphInstantiate(&b->exec, g, 0));
  return EHDG_OK;
}

// One graph with the batched loop. The looped instances' step is a handful
// of launches for all of them together: reset, right-hand side, initial
// trace, work lists and the first FP64 sweep; one WHILE node whose body is
// the batched loop (corrections, update, FP64 sweep over every instance that
// still iterates); reconstruction, trace hand-over and step record. Instances
// the loop does not take run their whole steps (each with its own loop) on
// the graph's branches, concurrently with all of it.
static ehdg_status batch_build_graph(ehdg_batch b) {
  const int n = (int)b->inst.size();
  b->looped.assign(n, 0);
  int n_loop = 0;
  for (int i = 0; i < n && b->use_loop; ++i) {
    const Ctx& c = b->inst[i]->c;
    if (!batch_loop_ok(c) || c.have_force) continue;
    b->looped[i] = 1;
    ++n_loop;
  }
  if (n_loop == 0 || n_loop > 8192) {   // the loop's list builder scans the instances in
    b->loop.release();                   // one block
    return batch_build_graph_branches(b);
  }
  batch_destroy_graph(b);
  const int k = std::min(n, b->chains > 0 ? b->chains : hw_queues());
  bool estimated = false;
  const std::vector<std::vector<int>> lists = batch_schedule(b, k, &estimated);
  std::vector<Ctx*> ctxs;
  std::vector<int> slots;
  for (int i = 0; i < n; ++i)
    if (b->looped[i]) {
      ctxs.push_back(&b->inst[i]->c);
      slots.push_back(i);
    }
  CK(b->loop.build(ctxs, b->t_start, b->t_acc, b->t_conv, slots));
  std::vector<cudaEvent_t> evs;
  auto event = [&](cudaEvent_t* e) {
    const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (r == cudaSuccess) evs.push_back(*e);
    return r;
  };
  auto cleanup_events = [&]() {
    for (auto e : evs) cudaEventDestroy(e);
  };
  cudaEvent_t fork = nullptr;
  if (event(&fork) != cudaSuccess) {
    cleanup_events();
    return cuda_fail(cudaGetLastError(), "batch events");
  }
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cleanup_events();
    return cuda_fail(e, "batch capture");
  }
  std::vector<cudaStream_t> forked;       // branches to join back before the end
  ehdg_status st = EHDG_OK;
  auto join_all = [&]() {
    for (cudaStream_t x : forked) {
      cudaEvent_t j = nullptr;
      if (event(&j) != cudaSuccess) continue;
      cudaEventRecord(j, x);
      cudaStreamWaitEvent(b->cap, j, 0);
    }
    forked.clear();
  };
  e = cudaEventRecord(fork, b->cap);
  // instances outside the loop: their whole steps on the branches
  for (int j = 0; j < k && e == cudaSuccess && st == EHDG_OK; ++j) {
    bool any = false;
    for (int i : lists[j]) any = any || !b->looped[i];
    if (!any) continue;
    cudaStream_t s = b->branch[j];
    if ((e = cudaStreamWaitEvent(s, fork, 0)) != cudaSuccess) break;
    forked.push_back(s);
    for (int i : lists[j]) {
      if (b->looped[i]) continue;
      Ctx& c = b->inst[i]->c;
      if ((e = launch_stamp(s, b->t_start, b->t_acc, i, 0)) != cudaSuccess) break;
      if ((st = capture_step(c, s, b->body, false)) != EHDG_OK) break;
      if ((e = launch_stamp(s, b->t_start, b->t_acc, i, 1)) != cudaSuccess) break;
    }
  }
  // the looped instances in the persistent form: before the loop, one launch
  // for every iteration, after it
  const bool persist = b->use_persist && b->loop.persist_ok();
  if (e == cudaSuccess && st == EHDG_OK && persist) {
    e = b->loop.launch_pre(b->cap, 0, 0);
    if (e == cudaSuccess) e = b->loop.launch_persist(b->cap);
    if (e == cudaSuccess) e = b->loop.launch_post(b->cap);
  }
  // the looped instances: before the loop, the loop, after it
  if (e == cudaSuccess && st == EHDG_OK && !persist) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle handle;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(b->cap, &cst, nullptr, &g, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = b->loop.launch_pre(b->cap, handle);
    if (e == cudaSuccess)
      e = cudaStreamGetCaptureInfo(b->cap, &cst, nullptr, &g, &deps, nullptr, &ndeps);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cond;
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cond, g, deps, nullptr, ndeps, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(b->cap, &cond, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(b->body, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        const cudaError_t e2 = b->loop.launch_body(b->body, handle);
        const cudaError_t e3 = cudaStreamEndCapture(b->body, &body);
        e = e2 != cudaSuccess ? e2 : e3;
      }
    }
    if (e == cudaSuccess) e = b->loop.launch_post(b->cap);
  }
  if (e != cudaSuccess || st != EHDG_OK) {
    const std::string msg = e != cudaSuccess ? std::string("batch capture: ") + cudaGetErrorString(e)
                                             : g_err;
    join_all();
    abort_capture(b->cap);
    cleanup_events();
    g_err = msg;
    return st != EHDG_OK ? st : EHDG_ERR_CUDA;
  }
  join_all();
  for (int i = 0; i < n; ++i) {
    b->graph_force[i] = b->inst[i]->c.have_force ? 1 : 0;
    b->graph_gen[i] = b->inst[i]->c.path_gen;
  }
  b->built_on_estimate = estimated;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap, &g);
  cleanup_events();
  if (e != cudaSuccess) return cuda_fail(e, "batch end capture");
  b->graph = g;
  CK(cudaGraphInstantiate(&b->exec, g, 0));
  return EHDG_OK;
}

ehdg_status ehdg_batch_create(int n, const ehdg_mesh_desc* meshes, const ehdg_problem_desc* probs,
                              void* stream, ehdg_batch* out) {
  if (!out || n < 1 || !meshes || !probs) return fail(EHDG_ERR_INVALID, "bad batch arguments");
  *out = nullptr;
  ehdg_batch b = new (std::nothrow) ehdg_batch_s();
  if (!b) return fail(EHDG_ERR_OOM, "host allocation failed");
  b->stream = (cudaStream_t)stream;
  auto bail = [&](ehdg_status s) {
    const std::string msg = g_err;
    ehdg_batch_destroy(b);
    g_err = msg;
    return s;
  };
  for (int i = 0; i < n; ++i) {
    ehdg_ctx h = nullptr;
    const ehdg_status st = ehdg_create(&meshes[i], &probs[i], stream, &h);
    if (st != EHDG_OK) {
      g_err = "instance " + std::to_string(i) + ": " + g_err;
      return bail(st);
    }
    b->inst.push_back(h);
  }
  b->branch.resize(n, nullptr);
  for (int i = 0; i < n; ++i)
    if (cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) != cudaSuccess)
      return bail(cuda_fail(cudaGetLastError(), "branch stream"));
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->body, cudaStreamNonBlocking) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "capture stream"));
  if (cudaMalloc(&b->t_start, sizeof(unsigned long long) * n) != cudaSuccess ||
      cudaMalloc(&b->t_acc, sizeof(unsigned long long) * n) != cudaSuccess ||
      cudaMalloc(&b->t_conv, sizeof(unsigned long long) * n) != cudaSuccess)
    return bail(fail(EHDG_ERR_OOM, "cudaMalloc failed"));
  if (cudaMemset(b->t_conv, 0, sizeof(unsigned long long) * n) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "cudaMemset"));
  b->graph_force.assign(n, 0);
  b->graph_gen.assign(n, 0);
  *out = b;
  return EHDG_OK;
}

ehdg_status ehdg_batch_instance(ehdg_batch b, int i, ehdg_ctx* out) {
  if (!b || !out || i < 0 || i >= (int)b->inst.size()) return fail(EHDG_ERR_INVALID, "bad instance");
  *out = b->inst[i];
  return EHDG_OK;
}

ehdg_status ehdg_batch_run(ehdg_batch b, int n_steps, int* iters, double* inst_time_s) {
  if (!b || n_steps < 0) return fail(EHDG_ERR_INVALID, "bad argument");
  const int n = (int)b->inst.size();
  if (n_steps == 0) return EHDG_OK;
  if (!b->tuning) b->last_run_steps = n_steps;
  bool rebuild = !b->exec;
  for (int i = 0; i < n; ++i) {
    Ctx& c = b->inst[i]->c;
    const int cap = c.step_cap;
    TRY(ensure_step_arrays(c, n_steps));
    if (c.step_cap != cap || (c.have_force ? 1 : 0) != b->graph_force[i] ||
        c.path_gen != b->graph_gen[i])
      rebuild = true;
  }
  if (rebuild) TRY(batch_build_graph(b));
  // the instance contexts run on the batch's stream: order their earlier work first
  CK(cudaStreamSynchronize(b->stream));
  CK(cudaMemsetAsync(b->t_acc, 0, sizeof(unsigned long long) * n, b->stream));
  for (int i = 0; i < n; ++i)
    CK(cudaMemsetAsync(&b->inst[i]->c.it->step, 0, sizeof(int), b->stream));
  if (b->profiling && b->loop.impl) {
    // kernel accounting: the looped instances' steps driven from the host with
    // every launch timed, the other instances' steps by their own graphs
    for (int i = 0; i < n; ++i)
      if (!b->looped[i]) {
        Ctx& c = b->inst[i]->c;
        cudaStream_t own = c.stream;
        c.stream = b->stream;
        const ehdg_status st = run_graph(c, n_steps, nullptr, nullptr);
        c.stream = own;
        if (st != EHDG_OK && st != EHDG_ERR_NOT_CONVERGED && st != EHDG_ERR_DIVERGED) return st;
      }
    int max_iter = 1;
    for (int i = 0; i < n; ++i) max_iter = std::max(max_iter, b->inst[i]->c.max_iter);
    for (int s = 0; s < n_steps; ++s)
      CK(b->loop.run_step_profiled(b->stream, max_iter, b->prof_ms, b->prof_launches,
                                   b->use_persist));
  } else {
    for (int s = 0; s < n_steps; ++s) CK(cudaGraphLaunch(b->exec, b->stream));
  }
  std::vector<unsigned long long> acc(n);
  CK(cudaMemcpyAsync(acc.data(), b->t_acc, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost,
                     b->stream));
  // flags of tensor-core waits that gave up (read with the results)
  std::vector<int> tc_err(n, 0);
  for (int i = 0; i < n; ++i) {
    Ctx& c = b->inst[i]->c;
    if (c.tc_err && (c.mixed || c.use_ozaki))
      CK(cudaMemcpyAsync(&tc_err[i], c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  }
  ehdg_status first = EHDG_OK;
  for (int i = 0; i < n; ++i) {
    Ctx& c = b->inst[i]->c;
    c.step_iters_h.resize(n_steps);
    c.step_status_h.resize(n_steps);
    CK(cudaMemcpyAsync(c.step_iters_h.data(), c.step_iters, sizeof(int) * n_steps,
                       cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(c.step_status_h.data(), c.step_status, sizeof(int) * n_steps,
                       cudaMemcpyDeviceToHost, b->stream));
  }
  CK(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < n; ++i) {
    Ctx& c = b->inst[i]->c;
    for (int s = 0; s < n_steps; ++s) {
      if (iters) iters[(int64_t)i * n_steps + s] = c.step_iters_h[s];
      if (first == EHDG_OK && c.step_status_h[s] != EHDG_OK) {
        first = (ehdg_status)c.step_status_h[s];
        g_err = "instance " + std::to_string(i) + " step " + std::to_string(s) + ": status " +
                std::to_string(c.step_status_h[s]);
      }
    }
    c.last_iters = std::min(c.step_iters_h[n_steps - 1], c.max_iter);
    if (inst_time_s) inst_time_s[i] = (double)acc[i] * 1e-9;
  }
  for (int i = 0; i < n && first == EHDG_OK; ++i)
    if (tc_err[i]) first = fail(EHDG_ERR_TIMEOUT, "instance " + std::to_string(i) +
                                                      ": a sweep's bounded mbarrier wait gave up");
  // a schedule made on guessed iteration counts is made again on the
  // measured ones, once, before the next run
  if (first == EHDG_OK && b->built_on_estimate) TRY(batch_build_graph(b));
  return first;
}

ehdg_status ehdg_batch_set_profiling(ehdg_batch b, int on) {
  if (!b) return fail(EHDG_ERR_INVALID, "NULL batch");
  b->profiling = on != 0;
  for (int k = 0; k < EHDG_KERNEL_KINDS; ++k) {
    b->prof_ms[k] = 0.0;
    b->prof_launches[k] = 0;
  }
  return EHDG_OK;
}

ehdg_status ehdg_batch_kernel_stats(ehdg_batch b, int kind, int64_t* launches, double* total_ms) {
  if (!b || kind < 0 || kind >= EHDG_KERNEL_KINDS) return fail(EHDG_ERR_INVALID, "bad argument");
  if (launches) *launches = b->prof_launches[kind];
  if (total_ms) *total_ms = b->prof_ms[kind];
  return EHDG_OK;
}

ehdg_status ehdg_batch_set_loop(ehdg_batch b, int on) {
  if (!b || on < 0 || on > 2) return fail(EHDG_ERR_INVALID, "NULL batch or bad mode");
  if ((on != 0) != b->use_loop || (on == 2) != b->use_persist) {
    b->use_loop = on != 0;
    b->use_persist = on == 2;
    batch_destroy_graph(b);
  }
  return EHDG_OK;
}

ehdg_status ehdg_batch_set_chains(ehdg_batch b, int k) {
  if (!b) return fail(EHDG_ERR_INVALID, "NULL batch");
  if (k != b->chains) {
    b->chains = k;
    batch_destroy_graph(b);
  }
  return EHDG_OK;
}

}  // extern "C"

// One batch step (graph launch) from the instances' current states per
// variant (apply(k) configures variant k, false skips it), every state
// restored after each; ms[k] is the second of two steps (the first captures
// the graph), or 1e300 for a skipped variant.
template <class Apply>
static ehdg_status batch_time_variants(ehdg_batch b, int n, Apply apply, double* ms) {
  std::vector<std::pair<void*, size_t>> arrays;
  for (auto h : b->inst)
    for (auto& a : state_arrays(h->c)) arrays.push_back(a);
  std::vector<void*> snap(arrays.size(), nullptr);
  auto free_snap = [&]() {
    for (void* p : snap)
      if (p) cudaFree(p);
  };
  CK(cudaStreamSynchronize(b->stream));
  for (size_t i = 0; i < arrays.size(); ++i) {
    if (cudaMalloc(&snap[i], arrays[i].second) != cudaSuccess ||
        cudaMemcpyAsync(snap[i], arrays[i].first, arrays[i].second, cudaMemcpyDeviceToDevice,
                        b->stream) != cudaSuccess) {
      free_snap();
      return fail(EHDG_ERR_OOM, "batch autotune snapshot failed");
    }
  }
  auto restore = [&]() {
    for (size_t i = 0; i < arrays.size(); ++i)
      cudaMemcpyAsync(arrays[i].first, snap[i], arrays[i].second, cudaMemcpyDeviceToDevice,
                      b->stream);
    return cudaStreamSynchronize(b->stream);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ehdg_status st = EHDG_OK;
  // each candidate is timed over as many steps as the batch's last run (the
  // run the choice is for), or one step before the first run
  const int steps = b->last_run_steps > 0 ? b->last_run_steps : 1;
  b->tuning = true;
  for (int q = 0; q < n; ++q) {
    ms[q] = 1e300;
    if (st != EHDG_OK || !apply(q)) continue;
    for (int rep = 0; rep < 2 && st == EHDG_OK; ++rep) {
      if (rep == 0) batch_destroy_graph(b);
      cudaEventRecord(e0, b->stream);
      st = ehdg_batch_run(b, steps, nullptr, nullptr);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (restore() != cudaSuccess && st == EHDG_OK) st = cuda_fail(cudaGetLastError(), "restore");
      if (rep == 1 && st == EHDG_OK) ms[q] = t;
    }
  }
  b->tuning = false;
  free_snap();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_destroy_graph(b);
  return st;
}

static int fastest(const int* cands, const double* ms, int n, int fallback, double* best_ms) {
  int best = fallback;
  double t = 1e300;
  for (int q = 0; q < n; ++q)
    if (ms[q] < t) {
      t = ms[q];
      best = cands[q];
    }
  if (best_ms) *best_ms = t;
  return best;
}

extern "C" {

ehdg_status ehdg_batch_autotune_chains(ehdg_batch b, const int* cands, int n_cands, int* best,
                                       double* best_ms) {
  if (!b || !cands || n_cands < 1) return fail(EHDG_ERR_INVALID, "bad argument");
  const int saved = b->chains;
  std::vector<double> ms((size_t)n_cands);
  const ehdg_status st = batch_time_variants(
      b, n_cands,
      [&](int q) {
        b->chains = cands[q];
        return true;
      },
      ms.data());
  b->chains = (st == EHDG_OK) ? fastest(cands, ms.data(), n_cands, saved, best_ms) : saved;
  if (best) *best = b->chains;
  return st;
}

ehdg_status ehdg_batch_autotune_schedule(ehdg_batch b, const int* chain_cands, int n_cands,
                                         int* loop_on, int* chains, double* best_ms) {
  if (!b || !chain_cands || n_cands < 1) return fail(EHDG_ERR_INVALID, "bad argument");
  const bool saved_loop = b->use_loop, saved_persist = b->use_persist;
  const int saved_chains = b->chains;
  // the persistent form is a candidate only where it applies (the instances
  // the loop takes, FP64 or FP32 corrections, fitting its ring)
  std::vector<const Ctx*> looped;
  for (auto h : b->inst)
    if (batch_loop_ok(h->c) && !h->c.have_force) looped.push_back(&h->c);
  const bool persist_applies =
      !looped.empty() && looped.size() <= 8192 && batch_persist_fits(looped);
  // variant 0: the batched loop, 1: its persistent form (branches keep the
  // current count); variant q >= 2: every instance on the branches,
  // chain_cands[q - 2] of them
  std::vector<double> ms((size_t)n_cands + 2);
  const ehdg_status st = batch_time_variants(
      b, n_cands + 2,
      [&](int q) {
        if (q >= 2 && chain_cands[q - 2] < 1) return false;
        if (q == 1 && !persist_applies) return false;
        b->use_loop = q < 2;
        b->use_persist = q == 1;
        if (q >= 2) b->chains = chain_cands[q - 2];
        return true;
      },
      ms.data());
  int best = -1;
  double t = 1e300;
  if (st == EHDG_OK)
    for (int q = 0; q < n_cands + 2; ++q)
      if (ms[q] < t) {
        t = ms[q];
        best = q;
      }
  if (best < 0) {
    b->use_loop = saved_loop;
    b->use_persist = saved_persist;
    b->chains = saved_chains;
  } else {
    b->use_loop = best < 2;
    b->use_persist = best == 1;
    b->chains = best < 2 ? saved_chains : chain_cands[best - 2];
  }
  batch_destroy_graph(b);
  if (loop_on) *loop_on = b->use_loop ? (b->use_persist ? 2 : 1) : 0;
  if (chains) *chains = b->chains;
  if (best_ms) *best_ms = t;
  return st;
}

ehdg_status ehdg_batch_autotune_inner_sweeps(ehdg_batch b, const int* cands, int n_cands,
                                             int* best, double* best_ms) {
  if (!b || !cands || n_cands < 1) return fail(EHDG_ERR_INVALID, "bad argument");
  const int n = (int)b->inst.size();
  std::vector<int> saved(n);
  int n_mixed = 0;
  for (int i = 0; i < n; ++i) {
    saved[i] = b->inst[i]->c.inner_sweeps;
    n_mixed += b->inst[i]->c.mixed ? 1 : 0;
  }
  if (n_mixed == 0) return fail(EHDG_ERR_INVALID, "no instance is mixed precision");
  // the inner sweep count is captured into each mixed instance's step graph
  auto set_all = [&](int m) {
    for (auto h : b->inst)
      if (h->c.mixed && h->c.inner_sweeps != m) {
        h->c.inner_sweeps = m;
        ++h->c.path_gen;
      }
  };
  std::vector<double> ms((size_t)n_cands);
  const ehdg_status st = batch_time_variants(
      b, n_cands,
      [&](int q) {
        if (cands[q] < 1 || cands[q] > 64) return false;
        set_all(cands[q]);
        return true;
      },
      ms.data());
  if (st == EHDG_OK) {
    const int m = fastest(cands, ms.data(), n_cands, -1, best_ms);
    if (m > 0) set_all(m);
    if (best) *best = m;
  } else {
    for (int i = 0; i < n; ++i) {
      ++b->inst[i]->c.path_gen;
      b->inst[i]->c.inner_sweeps = saved[i];
    }
  }
  return st;
}

ehdg_status ehdg_batch_autotune_sweep_tile(ehdg_batch b, const int* cands, int n_cands, int* best,
                                           double* best_ms) {
  if (!b || !cands || n_cands < 1) return fail(EHDG_ERR_INVALID, "bad argument");
  const int n = (int)b->inst.size();
  std::vector<int> saved(n);
  for (int i = 0; i < n; ++i) saved[i] = b->inst[i]->c.sweep_ft;
  auto set_all = [&](int ft) {
    for (auto h : b->inst) {
      if (h->c.sweep_ft != ft) ++h->c.path_gen;
      h->c.sweep_ft = ft;
    }
  };
  std::vector<double> ms((size_t)n_cands);
  const ehdg_status st = batch_time_variants(
      b, n_cands,
      [&](int q) {
        if (cands[q] != 2 && cands[q] != 4 && cands[q] != 8) return false;
        set_all(cands[q]);
        return true;
      },
      ms.data());
  if (st == EHDG_OK) {
    const int ft = fastest(cands, ms.data(), n_cands, saved[0], best_ms);
    set_all(ft);
    if (best) *best = ft;
  } else {
    for (int i = 0; i < n; ++i) {
      ++b->inst[i]->c.path_gen;
      b->inst[i]->c.sweep_ft = saved[i];
    }
  }
  return st;
}

void ehdg_batch_destroy(ehdg_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_destroy_graph(b);
  for (auto s : b->branch)
    if (s) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->body) cudaStreamDestroy(b->body);
  if (b->t_start) cudaFree(b->t_start);
  if (b->t_acc) cudaFree(b->t_acc);
  if (b->t_conv) cudaFree(b->t_conv);
  b->loop.release();
  for (auto h : b->inst) ehdg_destroy(h);
  delete b;
}

}  // extern "C"
