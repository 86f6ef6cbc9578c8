#!/usr/bin/env python
"""Benchmark of the eHDG hot path: trace DOF-iterations per second.

Workload (default): 2D transport on 256 x 256 quads, p = 4, per-element
velocity 0.5 (cos 2 pi y, sin 2 pi x) plus 8 seeded Fourier modes (amplitude
0.05), Crank-Nicolson dt = 2e-3 for 50 steps, eHDG to a trace residual of
1e-10 in every step, float64. One benchmark step = one full 50-step run from
the initial condition (set state + 50 implicit steps), i.e. one pass of the
whole hot path (per-step right-hand side, element sweeps, trace updates,
residual reductions, end-of-step reconstruction).

value: trace DOF x eHDG iterations / device time, inputs resident in HBM.
e2e:   the same through the C ABI with host buffers (state, boundary data in;
       state and trace out) inside the timed region.
--impl reference: the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# hardware work queues for concurrent graph branches (the batch workload);
# read when the CUDA context is created, so set before anything touches CUDA
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

METRIC = "trace DOF-iterations/s"
# GB300 FP64 FMA peak (CUDA cores): 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
UNIT = "DOF*iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="mesh side (256 is the benchmark size)")
    ap.add_argument("--time-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--workload", default="transport2d_varbeta",
                    choices=["transport2d_varbeta", "transport3d", "sw2d", "transport2d_small",
                             "steady2d", "batch", "residual"],
                    help="transport2d_varbeta is the benchmark; the others print a "
                         "time-to-tolerance comparison of FP64 and mixed precision")
    ap.add_argument("--inner-sweeps", type=int, default=8,
                    help="inner sweeps m of mixed precision (the benchmark workload tunes m "
                         "per precision unless --no-tune-inner)")
    ap.add_argument("--no-tune-inner", dest="tune_inner", action="store_false")
    ap.add_argument("--host-loop", action="store_true",
                    help="comparison workloads: host-driven steps (one launch per kernel, "
                         "visible to ncu) instead of graph-launched steps")
    ap.add_argument("--n-inst", type=int, default=256)
    ap.add_argument("--batch-chains", type=int, default=0,
                    help="batch workload: fixed graph branch count k instead of "
                         "ehdg_batch_autotune_chains")
    return ap.parse_args()


def workload(n, n_steps):
    from paper_1601_06681_gb300 import workloads as W
    return W.transport_2d_variable(n=(n, n), p=4, dt=2e-3, n_steps=n_steps, tol=1e-10)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(ms, units, ws, device=None):
    """Whole-job figures of ws independent replicas: the slowest rank's timed
    milliseconds, the units all ranks processed, and their throughput."""
    if ws <= 1:
        return ms, units, units / (ms * 1e-3)
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(u, op=torch.distributed.ReduceOp.SUM)
    t_max, u_all = float(t.item()), float(u.item())
    return t_max, u_all, u_all / (t_max * 1e-3)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_sha(sources):
    """sha256[:16] of the concatenated source files (paths under csrc/)."""
    import hashlib
    h = hashlib.sha256()
    for s in sources:
        with open(os.path.join(ROOT, "paper_1601_06681_gb300", "csrc", s), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


SWEEP_SOURCES = ("sweep_tiled.cu", "sweep_pass.cuh", "tiled_common.cuh", "sweep_common.cuh")


def kernel_traffic(kernel, sources):
    """DRAM bytes per sweep from the committed ncu summary, if the kernel's
    source files are unchanged since it was captured (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    ent = d.get(kernel)
    if not ent:
        return None
    return ent["bytes_per_sweep"] if ent.get("source_sha") == source_sha(sources) else None


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample(n_side=32, n_time=2, repeats=1):
    """Oracle throughput on a n_side x n_side corner of the benchmark mesh
    (same element size 1/256, velocity field, p, dt, scheme), n_time steps."""
    from oracle.ehdg import Problem
    from oracle.geometry import face_point_coords, node_coords
    from paper_1601_06681_gb300 import workloads as W
    wl = workload(256, n_time)
    h = 1.0 / 256
    mesh = W.structured_mesh((n_side, n_side), lo=[0.0, 0.0], hi=[n_side * h, n_side * h])
    X = node_coords(mesh, wl.p)
    prob = Problem(mesh, wl.p, scheme="cn", dt=wl.dt, beta_nodes=wl.beta_nodes(X))
    XF = face_point_coords(mesh, wl.p, prob.ref.q)
    u0 = wl.initial(X)
    g = wl.boundary(XF, 0.0)
    trace_dof = mesh["n_face"] * (wl.p + 1)
    times, units = [], []
    for _ in range(repeats):
        t0 = time.perf_counter()
        _, _, iters, _ = prob.run(u0, n_time, g_of_t=lambda t: g, tol=wl.tol)
        times.append(time.perf_counter() - t0)
        units.append(trace_dof * sum(iters))
    return times, units, f"{n_side}x{n_side} corner of the 256x256 mesh, {n_time} CN steps"


def _oracle_worker_init():
    # import the oracle before the timed map
    import oracle.ehdg  # noqa: F401
    import oracle.geometry  # noqa: F401


def _oracle_worker(args):
    n_side, n_time = args
    times, units, _ = oracle_sample(n_side, n_time, repeats=1)
    return times[0], units[0]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle, as it stands, on every host core: one process per core
    (spawned, single-threaded BLAS), each running its own corner sample."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init)

    def run(self, n_side=32, n_time=2):
        """(wall s, units, sample) of one round: every core runs one sample."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(n_side, n_time)] * self.cores, chunksize=1)
        wall = time.perf_counter() - t0
        return wall, sum(u for _, u in res), (
            f"{self.cores} processes, one per host core, each the oracle on a {n_side}x{n_side} "
            f"corner of the 256x256 mesh, {n_time} CN steps")

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    pool = OraclePool()
    for _ in range(max(args.warmup, 0)):
        pool.run()
    walls, units = [], []
    for _ in range(args.steps):
        w, u, sample = pool.run()
        walls.append(w)
        units.append(u)
    pool.close()
    value = sum(units) / sum(walls)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "transport2d_varbeta_256x256_p4_cn (oracle sample)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_1601_06681_gb300 import build, ehdg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build()
    ehdg.load()

    wl = workload(args.n, args.time_steps)
    mesh = ehdg.ehdg_mesh_structured((args.n, args.n))
    stream = torch.cuda.current_stream()
    # node coordinates come from the library (inputs are evaluated there)
    probe = None
    t_setup0 = time.perf_counter()
    solver = ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=wl.tol, max_iter=200,
                         beta_nodes=_beta_nodes(ehdg, mesh, wl), stream=stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup0
    X = solver.node_coords()
    XF = solver.face_point_coords()
    u0_h = np.ascontiguousarray(wl.initial(X))
    g_h = np.ascontiguousarray(wl.boundary(XF, 0.0))
    u0_d = torch.from_numpy(u0_h).to(dev)
    g_d = torch.from_numpy(g_h).to(dev)
    solver.set_boundary(g_d)
    trace_dof = solver.info["n_face"] * (wl.p + 1)

    def one_run():
        solver.set_state(u0_d)
        return solver.run(wl.n_steps)

    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    # timed region: graph-launched steps (device-side convergence loop)
    solver.set_profiling(False)          # resets the launch counters
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters_total = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            iters_total += sum(one_run())
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launch_counts = solver.kernel_stats()
    t_max, _, value = combine_ranks(ms, trace_dof * iters_total, ws, dev)

    # per-kernel device time: the same run with every launch bracketed by
    # CUDA events on the library's stream (host-driven loop, same kernels)
    solver.set_profiling(True)
    prof_sweeps = sum(one_run())
    stats = solver.kernel_stats()
    solver.set_profiling(False)

    # mixed precision on the same workload: time to the same FP64 tolerance,
    # with FP32 and with BF16 copies of the operator for the correction sweeps
    u_fp64, _ = solver.get_state()
    mixed = None
    if not args.no_mixed:
        mixed = {"fp64_ms_per_run": t_max / args.steps}
        for prec in ("fp32", "bf16"):
            ms_solver = ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=wl.tol,
                                    max_iter=200, beta_nodes=_beta_nodes(ehdg, mesh, wl),
                                    precision=prec, inner_sweeps=args.inner_sweeps, stream=stream)
            ms_solver.set_boundary(g_d)
            ms_solver.set_state(u0_d)
            # the inner sweep count m from ehdg_autotune_inner_sweeps (one timed
            # step per candidate from the initial state, which is restored)
            m_best = args.inner_sweeps
            if args.tune_inner:
                m_best, _ = ms_solver.autotune_inner_sweeps((4, 6, 8, 12, 16, 24))
            ms_solver.run(wl.n_steps)                      # warm-up
            torch.cuda.synchronize()
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            mit = 0
            for _ in range(args.steps):
                ms_solver.set_state(u0_d)
                mit += sum(ms_solver.run(wl.n_steps))
            m1.record(stream)
            torch.cuda.synchronize()
            mms = m0.elapsed_time(m1) / args.steps
            u_mx, _ = ms_solver.get_state()
            mixed[prec] = {
                "precision": f"{prec} operator in the correction sweeps (FP32 arithmetic) "
                             "+ fp64 defect correction",
                "inner_sweeps": m_best,
                "ms_per_run": mms, "speedup_time_to_tol": (t_max / args.steps) / mms,
                "fp64_sweeps_per_run": mit / args.steps,
                "rel_l2_vs_fp64": float(np.linalg.norm(u_mx - u_fp64) / np.linalg.norm(u_fp64))}
            ms_solver.close()

    # end to end through host buffers: inputs and outputs in pinned host memory
    # (the library copies through its own staging buffer with cudaMemcpyAsync)
    g_pin = torch.from_numpy(g_h).pin_memory()
    u0_pin = torch.from_numpy(u0_h).pin_memory()
    u_pin = torch.empty(solver.state_shape, dtype=torch.float64).pin_memory()
    uh_pin = torch.empty(solver.trace_shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    it_e2e = 0
    for _ in range(args.steps):
        solver.set_boundary(g_pin)
        solver.set_state(u0_pin)
        it_e2e += sum(solver.run(wl.n_steps))
        solver.get_state(u_pin, uh_pin)
    torch.cuda.synchronize()
    u_out, uh_out = u_pin.numpy(), uh_pin.numpy()
    e_s = time.perf_counter() - e0
    _, _, e2e_value = combine_ranks(e_s * 1e3, trace_dof * it_e2e, ws, dev)

    # roofline of the dominant kernel (the element sweep: k_sweep_persist, the
    # persistent form of k_sweep_tiled that runs a step's iterations in one
    # launch; figures are per sweep = per iteration): per
    # element and sweep it reads its operator rows (rows x NQFS doubles), Gy
    # and the point id of each row, the trace at its NQFS face points, its 4
    # face ids and face Jacobians and its two row counts, and writes one value
    # per row; flops = 2 x rows x NQFS
    # one launch of the element sweep runs either one iteration or (the
    # persistent form) every iteration of a step: time per sweep = total
    # sweep time / iterations
    n_elem_launch, elem_ms = stats["elem"]
    info = solver.info
    nq = 4 * info["Nqf"]
    rows = info["sweep_rows"]
    alg_bytes = (8 * rows * (nq + 2) + rows + 8 * nq * info["n_elem"]
                 + (4 * 4 + 4 * 8 + 2) * info["n_elem"])
    avg_ms = elem_ms / max(prof_sweeps, 1)
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    flops_per_launch = 2.0 * nq * rows
    launches = sum(v[0] for v in launch_counts.values())
    share = {k: round(v[1] / max(sum(x[1] for x in stats.values()), 1e-12), 4) for k, v in stats.items()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"transport2d_varbeta_{args.n}x{args.n}_p4_cn",
                       "n_elem": info["n_elem"], "p": wl.p, "time_steps_per_run": wl.n_steps,
                       "dt": wl.dt, "tol": wl.tol, "trace_dof": trace_dof,
                       "iterations_per_run": iters_total / args.steps,
                       "l2": "inputs larger than L2 (per-element operators "
                             f"{info['device_bytes'] / 1e9:.2f} GB resident)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "setup_s": round(setup_s, 3)},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(u0_h.nbytes + g_h.nbytes),
                    "d2h_bytes_per_step": int(u_out.nbytes + uh_out.nbytes)},
            "gpu_launches": int(launches),
            "roofline": {"kernel": "k_sweep_persist", "bound": "alu",
                         "achieved": flops_per_launch / (avg_ms * 1e-3) / 1e12,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops_per_launch / (avg_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz "
                                        "(FMA-chain probe measured 1.30 TFLOP/s)",
                         "traffic": kernel_traffic("k_sweep_persist", SWEEP_SOURCES),
                         "alg_bytes_per_sweep": alg_bytes,
                         "flops_per_sweep": flops_per_launch,
                         "avg_sweep_us": avg_ms * 1e3,
                         "sweep_launches": int(n_elem_launch), "sweeps": int(prof_sweeps),
                         "hbm_view": {"achieved_gbs": achieved, "peak_gbs": peak,
                                      "frac": achieved / peak, "peak_source": peak_src}},
            "kernel_time_share": share,
            "mixed_precision": mixed,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            # the oracle on every host core (a warm-up round, then a timed one),
            # and on one core
            pool = OraclePool()
            pool.run()
            wall, cu_all, sample_all = pool.run()
            pool.close()
            times, cu, sample = oracle_sample(repeats=1)
            line["cpu_baseline"] = {"value": cu_all / wall, "unit": UNIT, "cores": pool.cores,
                                    "kind": "oracle", "sample": sample_all,
                                    "value_one_core": sum(cu) / sum(times),
                                    "sample_one_core": sample}
        print(json.dumps(line), flush=True)
    solver.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def _beta_nodes(ehdg, mesh, wl):
    """Nodal velocity [n_elem][2][Np] at the library's own node coordinates."""
    # a throwaway constant-velocity context gives the node coordinates
    tmp = ehdg.Solver(mesh, wl.p, scheme="be", dt=1.0, beta_const=[1.0, 0.0], max_iter=1)
    X = tmp.node_coords()
    tmp.close()
    return wl.beta_nodes(X)


# ---------------------------------------------------------------------------
# other workloads: FP64 versus mixed precision, time to the same tolerance
# ---------------------------------------------------------------------------
def compare_workload(args):
    import torch
    from paper_1601_06681_gb300 import build, ehdg
    from paper_1601_06681_gb300 import workloads as W
    torch.cuda.set_device(0)
    build.build()
    ehdg.load()
    stream = torch.cuda.current_stream()
    if args.workload == "transport3d":
        wl = W.transport_3d(n=(args.n, args.n, args.n), p=3, n_steps=args.time_steps)
        precisions = ["fp64", "fp64+tiles", "fp64_emulated", "tf32", "bf16", "fp32",
                      "bf16+emulated_outer"]
    elif args.workload == "sw2d":
        # dt at which Theorem 2 holds on this mesh: h / (dt (p+1)(p+2)) = 3.9, C = 0.34
        wl = W.sw_2d(n=(args.n, args.n), p=3, dt=2.5e-5, n_steps=args.time_steps)
        precisions = ["fp64", "fp64_emulated", "tf32", "bf16", "fp32", "bf16+emulated_outer"]
    elif args.workload == "steady2d":
        # the steady solve of Sec. 4.1 (one "step", many iterations)
        wl = W.steady_2d_smooth(n=(args.n, args.n), p=4)
        precisions = ["fp64", "fp32", "bf16"]
    else:
        wl = W.transport_2d_small(n=(args.n, args.n), p=2, n_steps=args.time_steps)
        precisions = ["fp64", "fp64+tiles", "fp64_emulated", "tf32", "fp32"]
    mesh = ehdg.ehdg_mesh_structured(wl.n, boundary_tag=(2 if wl.pde == "sw" else 1))
    results = {}
    ref = None
    for prec in precisions:
        # "<precision>+emulated_outer": mixed precision whose outer FP64 sweeps
        # run FP64-accurate on the tensor cores; "+tiles": the fused sweep's
        # tile shape from ehdg_autotune_sweep_tile
        base, _, opt = prec.partition("+")
        kw = dict(pde=wl.pde, scheme=wl.scheme, dt=wl.dt, tol=wl.tol,
                  max_iter=20000 if wl.scheme == "steady" else 400,
                  precision=base, inner_sweeps=args.inner_sweeps, stream=stream,
                  emulated_outer=(opt == "emulated_outer"))
        if wl.pde == "sw":
            kw["Phi"] = wl.Phi
        elif wl.beta_fn is not None:
            kw["beta_nodes"] = _beta_nodes(ehdg, mesh, wl)
        else:
            kw["beta_const"] = wl.beta_const
        s = ehdg.Solver(mesh, wl.p, **kw)
        if args.host_loop:
            s.set_profiling(True)       # ehdg_step then drives the loop from the host
        X, XF = s.node_coords(), s.face_point_coords()
        u0 = torch.from_numpy(np.ascontiguousarray(wl.initial(X))).cuda()
        gs = [torch.from_numpy(np.ascontiguousarray(wl.boundary(XF, k * wl.dt))).cuda()
              for k in range(wl.n_steps + 1)]
        f_nodes = wl.forcing(X)
        if f_nodes is not None:
            s.set_forcing(np.ascontiguousarray(f_nodes))
        tile_ft = None
        if opt == "tiles":
            s.set_boundary(gs[0])
            s.set_state(u0)
            tile_ft = s.autotune_sweep_tile()[0]
        m_best = None
        if base in ("tf32", "bf16", "fp32") and args.tune_inner:
            # inner sweep count from ehdg_autotune_inner_sweeps (state restored)
            s.set_boundary(gs[0])
            s.set_state(u0)
            m_best = s.autotune_inner_sweeps((4, 6, 8, 12, 16, 24))[0]

        def one_run():
            # graph-launched steps (the device-side loop); a transport step
            # takes that step's inflow data first, so one graph launch per step
            s.set_boundary(gs[0])
            s.set_state(u0)
            if wl.pde == "sw" and not args.host_loop:
                return sum(s.run(wl.n_steps))
            its = 0
            for k in range(wl.n_steps):
                if wl.pde != "sw":
                    s.set_boundary(gs[k + 1])
                its += s.step()[0] if args.host_loop else s.run(1)[0]
            return its

        one_run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = 0
        for _ in range(args.steps):
            its = one_run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        u, _ = s.get_state()
        if ref is None:
            ref = u
        results[prec] = {"ms_per_run": ms, "fp64_sweeps_per_run": its,
                         "rel_l2_vs_fp64": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
                         "speedup_vs_fp64": None}
        if tile_ft is not None:
            results[prec]["tile_ft"] = tile_ft
        if m_best is not None:
            results[prec]["inner_sweeps"] = m_best
        if "exact" in wl.meta:
            ue = wl.meta["exact"](X)[:, None, :]
            results[prec]["max_nodal_error_vs_exact"] = float(np.max(np.abs(u - ue)))
        s.close()
    for prec in precisions:
        results[prec]["speedup_vs_fp64"] = results["fp64"]["ms_per_run"] / results[prec]["ms_per_run"]
    info = {"workload": wl.name, "n_elem": int(np.prod(wl.n)), "p": wl.p, "dt": wl.dt,
            "time_steps": wl.n_steps, "tol": wl.tol,
            "inner_sweeps": "tuned per precision" if args.tune_inner else args.inner_sweeps}
    print(json.dumps({"metric": "time-to-tol per run, mixed vs FP64", "config": info,
                      "results": results}), flush=True)


def residual_workload(args):
    """The standalone FP64 trace-residual reduction sqrt(sum w (a - b)^2)
    (the convergence check of Algorithm 1) on 2^24 face points, 402.7 MB
    read per call, larger than L2: HBM rate against the copy peak."""
    import torch
    from paper_1601_06681_gb300 import build, ehdg
    torch.cuda.set_device(0)
    build.build()
    ehdg.load()
    stream = torch.cuda.current_stream()
    n = 1 << 24
    g = torch.Generator(device="cuda")
    g.manual_seed(1005)
    a = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    b = a + 1e-6 * torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    w = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    res = {}
    for name, fn in (("ehdg_trace_residual", ehdg.ehdg_trace_residual),
                     ("ehdg_trace_residual_noalloc", ehdg.ehdg_trace_residual_noalloc)):
        for _ in range(max(args.warmup, 3)):
            fn(a, b, w, out, stream)
        torch.cuda.synchronize()
        reps = 50
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn(a, b, w, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = 1e3 * e0.elapsed_time(e1) / reps
        gbs = 3 * 8 * n / (us * 1e-6) / 1e9
        ref = float(torch.sqrt(torch.sum(w * (a - b) ** 2)))
        res[name] = {"us_per_call": us, "achieved_gbs": gbs, "frac_of_peak": gbs / peak,
                     "rel_err_vs_torch": abs(float(out.item()) - ref) / ref}
    print(json.dumps({"metric": "FP64 trace residual, HBM rate", "n_points": n,
                      "bytes_per_call": 3 * 8 * n, "peak_gbs": peak, "peak_source": peak_src,
                      "l2": "inputs larger than L2 (402.7 MB per call)", "results": res}),
          flush=True)


def batch_workload(args):
    """Config 5: independent 2D transport instances (N 8..128, p 1..5) stepped
    together, one graph launch per time step; FP64 versus mixed precision.
    Each variant's graph branch count comes from the batch autotuner (setup,
    outside the timed run)."""
    import torch
    from paper_1601_06681_gb300 import build, ehdg
    from paper_1601_06681_gb300 import workloads as W
    torch.cuda.set_device(0)
    build.build()
    ehdg.load()
    stream = torch.cuda.current_stream()
    wls = W.batched_mix(n_inst=args.n_inst)
    out = {}
    # "+tuned": every instance's FP64 path (DFMA or tensor cores) picked by
    # ehdg_autotune_fp64_path before the first run
    # "+tiles": the fused FP64 sweep's tile (row groups FT) of all instances
    # picked by ehdg_batch_autotune_sweep_tile before the first run
    variants = ["fp64", "tf32", "fp64_emulated", "tf32+emulated_outer", "fp64_emulated+tuned",
                "fp64+tiles", "tf32+tiles"]
    for prec in variants:
        base, _, opt = prec.partition("+")
        specs, inputs = [], []
        for wl in wls:
            mesh = ehdg.ehdg_mesh_structured(wl.n)
            specs.append(dict(mesh=mesh, p=wl.p, scheme=wl.scheme, dt=wl.dt, tol=wl.tol,
                              max_iter=400, beta_const=wl.beta_const, precision=base,
                              inner_sweeps=args.inner_sweeps,
                              emulated_outer=(opt == "emulated_outer")))
        t0 = time.perf_counter()
        b = ehdg.Batch(specs, stream=stream)
        setup = time.perf_counter() - t0
        for wl, s in zip(wls, b.instances):
            X, XF = s.node_coords(), s.face_point_coords()
            s.set_boundary(wl.u0_fn(XF))
            inputs.append(torch.from_numpy(np.ascontiguousarray(wl.initial(X))).cuda())
        n_tensor = None
        if opt == "tuned":
            n_tensor = 0
            for s, u0 in zip(b.instances, inputs):
                s.set_state(u0)
                n_tensor += int(s.autotune_fp64_path()[0])
        tile_ft = None
        if opt == "tiles":
            for s, u0 in zip(b.instances, inputs):
                s.set_state(u0)
            tile_ft, _ = b.autotune_sweep_tile()
        # the graph's branch count, picked by ehdg_batch_autotune_chains (or fixed)
        if args.batch_chains > 0:
            b.set_chains(args.batch_chains)
            chains = args.batch_chains
        else:
            for s, u0 in zip(b.instances, inputs):
                s.set_state(u0)
            chains, _ = b.autotune_chains()

        def one_run():
            for s, u0 in zip(b.instances, inputs):
                s.set_state(u0)
            return b.run(wls[0].n_steps)

        one_run()                                     # warm-up (captures the graph)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters, times = one_run()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[prec] = {"instances_per_s": len(wls) / wall, "wall_s": wall, "setup_s": setup,
                     "p50_instance_ms": float(np.percentile(times, 50) * 1e3),
                     "p99_instance_ms": float(np.percentile(times, 99) * 1e3),
                     "sweeps_total": int(iters.sum()), "chains": chains}
        if n_tensor is not None:
            out[prec]["instances_on_tensor_cores"] = n_tensor
        if tile_ft is not None:
            out[prec]["tile_ft"] = tile_ft
        b.close()
    for prec in variants[1:]:
        out[prec]["speedup_vs_fp64"] = out["fp64"]["wall_s"] / out[prec]["wall_s"]
    info = {"workload": f"batched_mix_{args.n_inst}", "time_steps": wls[0].n_steps,
            "elements_total": int(sum(np.prod(w.n) for w in wls))}
    print(json.dumps({"metric": "instances/s (one graph launch per step)", "config": info,
                      "results": out}), flush=True)


def main():
    args = parse()
    if args.workload == "residual":
        residual_workload(args)
        return
    if args.workload == "batch":
        batch_workload(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "transport2d_varbeta":
        compare_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
