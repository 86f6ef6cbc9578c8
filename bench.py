#!/usr/bin/env python
"""Benchmark of the eHDG hot path: trace DOF-iterations per second and
time to tolerance, mixed precision against FP64.

Headline workload (default): 3D scalar transport on 64^3 uniform hexahedra,
p = 3 (64 nodes per element), beta = (1,1,1)/sqrt(3), Gaussian initial data
(centre (0.3,0.3,0.3), sigma 0.08) plus seeded U(+-1e-3) noise, inflow data
from the advected Gaussian, backward Euler dt = 5e-3 for 20 steps, eHDG to a
trace residual of 1e-10 in every step. One benchmark step = one full 20-step
run from the initial condition (set state, then per implicit step: that
step's inflow data and one graph-launched step) -- one pass of the whole hot
path (per-step right-hand side, element sweeps with the fused trace update
and residual, end-of-step reconstruction).

value:       trace DOF x eHDG iterations / device time of the native FP64
             path (DFMA sweeps), inputs resident in HBM.
e2e:         the same through the C ABI with pinned host buffers (initial
             state, every step's boundary data in; state and trace out)
             inside the timed region.
time_to_tol: every path (FP64 on the DFMA pipe, FP64-accurate on the BF16
             tensor cores, TF32/BF16 corrections with FP64 defect correction)
             run to one stopping tolerance at which each lands within 1e-10
             relative L2 of the FP64 fixed point (the FP64 path converged to
             1e-13), with its time, speedup and distance to that fixed point,
             and the roofline of its dominant kernel.
secondary:   the 2D variable-velocity workload (256^2 quads, p = 4,
             per-element operators, Crank-Nicolson dt = 2e-3 x 50 steps).
shallow_water: linearised shallow water on 512^2 quads, p = 3 (one shared
             48 x 48 operator), time to a matched tolerance of every path.
batch:       the batched mix of 256 independent 2D transport instances
             (N 8..128, p 1..5, BE dt = 0.01 x 10 steps), instances/s with
             p50/p99 per-instance times and each variant's distance to the
             instances' FP64 fixed points, at a matched-accuracy tolerance.
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
UNIT = "DOF*iter/s"
# stopping tolerance of the accuracy-matched time-to-tolerance comparison on
# the 3D workload: the largest of 1e-11, 3e-12, 1e-12 at which the FP64 path's
# state lies within 1e-10 relative L2 of its fixed point (each entry's
# distance is measured and reported in the same run)
TOL_MATCHED_3D = 3e-12
INNER_GRID_3D = (8, 12, 16, 20, 24)     # mixed precision's inner sweep counts tried first
INNER_REFINE = 4                        # then at most this many steps of one from the best
ACCURACY_TARGET = 1e-10
# bytes one element moves per sweep of a shared-operator transport sweep in
# the A^{-1} form of the algorithmic-work count: 8 (n + 2 T_own), n = 64,
# T_own = 48 owned trace values (3D, p = 3)
ALG_BYTES_PER_ELEM_3D = 8 * (64 + 2 * 48)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=0,
                    help="mesh side (default: 64 for the 3D headline, 256 for 2D)")
    ap.add_argument("--time-steps", type=int, default=0,
                    help="implicit steps per run (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="headline: leave out the batched-mix key")
    ap.add_argument("--no-sw", action="store_true",
                    help="headline: leave out the shallow-water key")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "transport2d_varbeta", "transport3d", "sw2d",
                             "transport2d_small", "steady2d", "batch", "residual"],
                    help="headline is the benchmark (3D transport, with the 2D "
                         "variable-velocity workload as a secondary key); "
                         "transport2d_varbeta prints that workload's line alone; the "
                         "others print a time-to-tolerance comparison of FP64 and mixed "
                         "precision")
    ap.add_argument("--inner-sweeps", type=int, default=8,
                    help="inner sweeps m of mixed precision (the 2D variable-velocity "
                         "workload tunes m per precision unless --no-tune-inner)")
    ap.add_argument("--no-tune-inner", dest="tune_inner", action="store_false")
    ap.add_argument("--host-loop", action="store_true",
                    help="comparison workloads: host-driven steps (one launch per kernel, "
                         "visible to ncu) instead of graph-launched steps")
    ap.add_argument("--n-inst", type=int, default=256)
    ap.add_argument("--batch-chains", type=int, default=0,
                    help="batch workload: fixed graph branch count k instead of "
                         "ehdg_batch_autotune_chains")
    ap.add_argument("--batch-variants", default="",
                    help="batch workload: comma-separated subset of its variants "
                         "(default: all)")
    ap.add_argument("--batch-tol", type=float, default=0.0,
                    help="batch workload: stopping tolerance of every instance "
                         "(default: the matched-accuracy 3e-12)")
    return ap.parse_args()


def workload(n, n_steps):
    """The 2D variable-velocity workload (per-element operators, CN)."""
    from paper_1601_06681_gb300 import workloads as W
    return W.transport_2d_variable(n=(n, n), p=4, dt=2e-3, n_steps=n_steps, tol=1e-10)


def workload_3d(n, n_steps):
    """The headline 3D transport workload (one shared operator, BE)."""
    from paper_1601_06681_gb300 import workloads as W
    return W.transport_3d(n=(n, n, n), p=3, dt=5e-3, n_steps=n_steps, tol=1e-10)


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


def kernel_traffic(key):
    """DRAM bytes per launch (per sweep) of a kernel on a workload from the
    committed ncu summary, if the kernel's source files are unchanged since it
    was captured (else None). key = "<kernel>@<workload>"."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    ent = d.get(key)
    if not ent:
        return None
    if ent.get("source_sha") != source_sha(ent["sources"]):
        return None
    return ent["bytes_per_sweep"]


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
ORACLE_SAMPLE_3D = (8, 2)      # an 8^3 corner of the 64^3 mesh, 2 BE steps
ORACLE_SAMPLE_2D = (32, 2)     # a 32^2 corner of the 256^2 mesh, 2 CN steps


def oracle_sample_3d(n_side=8, n_time=2):
    """Oracle throughput on an n_side^3 corner of the 64^3 headline mesh (same
    element size 1/64, velocity, p, dt, scheme, tolerance, initial and inflow
    data), n_time steps: (seconds, DOF-iterations, description)."""
    from oracle.ehdg import Problem
    from oracle.geometry import face_point_coords, node_coords
    from paper_1601_06681_gb300 import workloads as W
    wl = workload_3d(64, n_time)
    h = 1.0 / 64
    mesh = W.structured_mesh((n_side,) * 3, lo=[0.0] * 3, hi=[n_side * h] * 3)
    X = node_coords(mesh, wl.p)
    prob = Problem(mesh, wl.p, scheme="be", dt=wl.dt, beta_const=wl.beta_const)
    XF = face_point_coords(mesh, wl.p, prob.ref.q)
    u0 = wl.initial(X)
    trace_dof = mesh["n_face"] * prob.ref.Nqf
    t0 = time.perf_counter()
    _, _, iters, _ = prob.run(u0, n_time, g_of_t=lambda t: wl.boundary(XF, t), tol=wl.tol)
    return (time.perf_counter() - t0, trace_dof * sum(iters),
            f"{n_side}^3 corner of the 64^3 mesh, {n_time} BE steps")


def oracle_sample_2d(n_side=32, n_time=2):
    """Oracle throughput on an n_side^2 corner of the 256^2 variable-velocity
    mesh (same element size 1/256, velocity field, p, dt, scheme), n_time steps."""
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
    t0 = time.perf_counter()
    _, _, iters, _ = prob.run(u0, n_time, g_of_t=lambda t: g, tol=wl.tol)
    return (time.perf_counter() - t0, trace_dof * sum(iters),
            f"{n_side}x{n_side} corner of the 256x256 mesh, {n_time} CN steps")


def _oracle_worker_init():
    # import the oracle before the timed map
    import oracle.ehdg  # noqa: F401
    import oracle.geometry  # noqa: F401


def _oracle_worker(args):
    kind, n_side, n_time = args
    fn = oracle_sample_3d if kind == "3d" else oracle_sample_2d
    secs, units, _ = fn(n_side, n_time)
    return secs, units


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

    def run(self, kind="3d", n_side=None, n_time=None):
        """(wall s, units, sample) of one round: every core runs one sample
        (default size: ORACLE_SAMPLE_3D / ORACLE_SAMPLE_2D)."""
        d_side, d_time = ORACLE_SAMPLE_3D if kind == "3d" else ORACLE_SAMPLE_2D
        n_side, n_time = n_side or d_side, n_time or d_time
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(kind, n_side, n_time)] * self.cores, chunksize=1)
        wall = time.perf_counter() - t0
        what = (f"{n_side}^3 corner of the 64^3 mesh, {n_time} BE steps" if kind == "3d" else
                f"{n_side}x{n_side} corner of the 256x256 mesh, {n_time} CN steps")
        return wall, sum(u for _, u in res), (
            f"{self.cores} processes, one per host core, each the oracle on a {what}")

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(kind="3d"):
    """The oracle on every host core (a warm-up round, then a timed one) and on
    one core."""
    pool = OraclePool()
    pool.run(kind)
    wall, units_all, sample_all = pool.run(kind)
    pool.close()
    fn = oracle_sample_3d if kind == "3d" else oracle_sample_2d
    secs, units, sample = fn(*(ORACLE_SAMPLE_3D if kind == "3d" else ORACLE_SAMPLE_2D))
    return {"value": units_all / wall, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": sample_all, "value_one_core": units / secs, "sample_one_core": sample}


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    kind = "2d" if args.workload == "transport2d_varbeta" else "3d"
    pool = OraclePool()
    for _ in range(max(args.warmup, 0)):
        pool.run(kind)
    walls, units = [], []
    for _ in range(args.steps):
        w, u, sample = pool.run(kind)
        walls.append(w)
        units.append(u)
    pool.close()
    value = sum(units) / sum(walls)
    name = ("transport2d_varbeta_256x256_p4_cn" if kind == "2d" else "transport3d_64x64x64_p3_be")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name, "sample": sample,
                   "measures": "the oracle on a bounded sample of this workload, its "
                               "DOF-iterations per second of host time"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def fp64_peak(ehdg, stream, sm_mhz):
    """FP64 FMA peak of the device: the larger of the FMA-chain probe measured
    now (ehdg_probe_fp64_rate) and SMs x 2 FP64 FMA per clock x 2 flop x the
    median SM clock sampled during the timed region."""
    sms, probe = ehdg.ehdg_probe_fp64_rate(stream)
    derived = None if not sm_mhz else sms * 2 * 2 * sm_mhz * 1e6 / 1e12
    if derived is not None and derived > probe:
        return derived, (f"derived: {sms} SMs x 2 FP64 FMA/clk x 2 flop x {sm_mhz:.0f} MHz "
                         f"(median SM clock of the timed region; FMA-chain probe measured "
                         f"{probe:.3f} TFLOP/s)"), probe, derived, sms
    return probe, (f"measured: FMA-chain probe (ehdg_probe_fp64_rate) on {sms} SMs, "
                   f"{probe:.3f} TFLOP/s" + (f"; derived {derived:.3f} TFLOP/s from the median "
                                             f"SM clock {sm_mhz:.0f} MHz" if derived else "")
                   ), probe, derived, sms


def events_ms(stream, fn, reps):
    """Device time of reps calls of fn, CUDA events on `stream` (ms per call)
    and the value of the last call."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def events_ms_each(stream, fn, reps):
    """Device time of each of reps calls of fn (CUDA events on `stream`, ms)
    and the value of the last call."""
    import torch
    out, times = None, []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, out


M_MIN, M_MAX = 1, 64           # the library's range of inner sweep counts


def fastest_m(cands, build, stream, timer=None, refine=0):
    """Inner sweep count of mixed precision whose whole run is fastest:
    build(m) -> (context, one_run); each candidate is timed over one run after
    a warm-up run (timer(run) -> ms; CUDA events on `stream` by default).
    With refine > 0 the search then steps by one from the fastest candidate
    (m - 1 and m + 1, then on in the direction that was faster) while that
    is faster, building at most `refine` more contexts: the run time moves in
    steps with m (the outer iteration count is an integer), so the best m can
    fall between grid points. Returns (context, one_run, m, {m: ms}) with the
    kept context open and the others closed."""
    if timer is None:
        def timer(run):
            return events_ms_each(stream, run, 1)[0][0]
    best, tried = None, {}

    def trial(m):
        nonlocal best
        ctx, run = build(m)
        run()                                               # warm-up (captures the graph)
        t = timer(run)
        tried[str(m)] = round(t, 2)
        if best is None or t < best[3]:
            if best is not None:
                best[0].close()
            best = (ctx, run, m, t)
            return True
        ctx.close()
        return False

    for m in cands:
        trial(m)
    if refine > 0 and best[2] is not None:
        left, step = refine, None
        while left > 0:
            centre = best[2]
            dirs = (step,) if step else (-1, 1)
            moved = None
            for d in dirs:
                m = centre + d
                if left == 0 or not (M_MIN <= m <= M_MAX) or str(m) in tried:
                    continue
                left -= 1
                if trial(m):
                    moved = d
                    break
            if moved is None:
                break
            step = moved
    return best[0], best[1], best[2], tried


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def kernel_shares(stats):
    tot = max(sum(v[1] for v in stats.values()), 1e-12)
    return {k: round(v[1] / tot, 4) for k, v in stats.items() if v[0] > 0}


def run_2d(args, ws, dev, stream, standalone=False):
    """The 2D variable-velocity workload (256^2, p = 4, per-element operators,
    CN dt = 2e-3 x 50 steps): FP64 DOF-iterations/s, the roofline of the
    persistent sweep, mixed precision (FP32 / BF16 operator copies) against
    FP64 at a matched tolerance, with each state's distance to the FP64 fixed
    point."""
    import torch
    from paper_1601_06681_gb300 import ehdg
    n = args.n or 256
    wl = workload(n, args.time_steps or 50)
    mesh = ehdg.ehdg_mesh_structured((n, n))
    beta = _beta_nodes(ehdg, mesh, wl)
    t_setup0 = time.perf_counter()
    solver = ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=wl.tol, max_iter=200,
                         beta_nodes=beta, stream=stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup0
    X = solver.node_coords()
    XF = solver.face_point_coords()
    u0_h = np.ascontiguousarray(wl.initial(X))
    g_h = np.ascontiguousarray(wl.boundary(XF, 0.0))
    u0_d = torch.from_numpy(u0_h).to(dev)
    g_d = torch.from_numpy(g_h).to(dev)
    trace_dof = solver.info["n_face"] * (wl.p + 1)

    def runner(s):
        def one_run():
            s.set_boundary(g_d)
            s.set_state(u0_d)
            return sum(s.run(wl.n_steps))
        return one_run

    one_run = runner(solver)
    for _ in range(max(args.warmup, 1)):
        one_run()
    if ws > 1:
        torch.distributed.barrier()
    solver.set_profiling(False)          # resets the launch counters
    reps = max(args.steps, 1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters_total = 0
    e0.record(stream)
    for _ in range(reps):
        iters_total += one_run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launch_counts = solver.kernel_stats()
    t_max, _, value = combine_ranks(ms, trace_dof * iters_total, ws, dev)
    u_fp64, _ = solver.get_state()
    # per-kernel device time: one run with every launch bracketed by events
    solver.set_profiling(True)
    prof_sweeps = one_run()
    stats = solver.kernel_stats()
    solver.set_profiling(False)

    # the FP64 fixed point of the same run (every step to 1e-13)
    fix = ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=1e-13, max_iter=400,
                      beta_nodes=beta, stream=stream)
    runner(fix)()
    u_fix, _ = fix.get_state()
    fix.close()

    mixed = None
    if not args.no_mixed:
        # matched accuracy: FP64 and both mixed paths stop at the largest of
        # the config's tolerance, 1e-11, 3e-12, 1e-12 at which FP64 lands within
        # ACCURACY_TARGET of its fixed point (at 1e-10 it ends 2.7e-10 away)
        tol_errs, tol_m, u_ref, fp64_ms = {}, None, None, None
        for t in (wl.tol, 1e-11, 3e-12, 1e-12):
            if t == wl.tol:
                err, ref = rel_l2(u_fp64, u_fix), None    # the timed run stopped at wl.tol
            else:
                ref = ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=t, max_iter=200,
                                  beta_nodes=beta, stream=stream)
                runner(ref)()                              # warm-up (captures the graph)
                err = rel_l2(ref.get_state()[0], u_fix)
            tol_errs[f"{t:g}"] = err
            if err <= ACCURACY_TARGET or t == 1e-12:
                tol_m = t
                if ref is None:
                    fp64_ms, u_ref = t_max / reps, u_fp64
                else:
                    fp64_ms, _ = events_ms(stream, runner(ref), reps)
                    u_ref = ref.get_state()[0]
                    ref.close()
                break
            if ref is not None:
                ref.close()
        mixed = {"tol": tol_m,
                 "tol_rule": f"the largest of {wl.tol:g}, 1e-11, 3e-12, 1e-12 at which FP64 lands "
                             f"within {ACCURACY_TARGET:g} relative L2 of its fixed point (every "
                             "step to 1e-13); FP64 and both mixed paths run to it",
                 "fp64_rel_l2_vs_fixed_point_by_tol": tol_errs,
                 "fp64_ms_per_run": fp64_ms,
                 "fp64_rel_l2_vs_fp64_fixed_point": tol_errs[f"{tol_m:g}"]}
        for prec in ("fp32", "bf16"):
            def build(m, prec=prec):
                sv = ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=tol_m,
                                 max_iter=200, beta_nodes=beta, precision=prec,
                                 inner_sweeps=m, stream=stream)
                return sv, runner(sv)
            cands = (4, 6, 8, 12, 16, 24) if args.tune_inner else (args.inner_sweeps,)
            ms_solver, mrun, m_best, tried = fastest_m(cands, build, stream,
                                                       refine=INNER_REFINE if args.tune_inner else 0)
            mms, mit = events_ms(stream, mrun, reps)
            u_mx, _ = ms_solver.get_state()
            mixed[prec] = {
                "precision": f"{prec} operator in the correction sweeps (FP32 arithmetic) "
                             "+ fp64 defect correction",
                "inner_sweeps": m_best, "inner_sweeps_tried_ms_per_run": tried,
                "ms_per_run": mms,
                "speedup_time_to_tol": fp64_ms / mms, "fp64_sweeps_per_run": mit,
                "rel_l2_vs_fp64": rel_l2(u_mx, u_ref),
                "rel_l2_vs_fp64_fixed_point": rel_l2(u_mx, u_fix)}
            ms_solver.close()

    # roofline of the dominant kernel (k_sweep_persist, the persistent form of
    # k_sweep_tiled that runs a step's iterations in one launch; figures per
    # sweep): per element and sweep it reads its operator rows (rows x NQFS
    # doubles), Gy and the point id of each row, the trace at its NQFS face
    # points, its 4 face ids and face Jacobians and its two row counts, and
    # writes one value per row; flops = 2 x rows x NQFS
    info = solver.info
    nq = 4 * info["Nqf"]
    rows = info["sweep_rows"]
    alg_bytes = (8 * rows * (nq + 2) + rows + 8 * nq * info["n_elem"]
                 + (4 * 4 + 4 * 8 + 2) * info["n_elem"])
    avg_ms = stats["elem"][1] / max(prof_sweeps, 1)
    flops = 2.0 * nq * rows
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {
        "workload": f"transport2d_varbeta_{n}x{n}_p4_cn", "value": value, "unit": UNIT,
        "ms_per_run": t_max / reps, "n_elem": info["n_elem"], "p": wl.p,
        "time_steps_per_run": wl.n_steps, "dt": wl.dt, "tol": wl.tol, "trace_dof": trace_dof,
        "trace_dof_definition": "n_face x (p+1); the library stores q = 7 Gauss points per "
                                "face for this per-node velocity (p+1 = 5 counted)",
        "iterations_per_run": iters_total / reps, "setup_s": round(setup_s, 3),
        "fp64_rel_l2_vs_fp64_fixed_point": rel_l2(u_fp64, u_fix),
        "roofline": {"kernel": "k_sweep_persist", "bound": "alu",
                     "achieved_tflops": flops / (avg_ms * 1e-3) / 1e12,
                     "flops_per_sweep": flops, "alg_bytes_per_sweep": alg_bytes,
                     "avg_sweep_us": avg_ms * 1e3, "sweeps": int(prof_sweeps),
                     "traffic": kernel_traffic(f"k_sweep_persist@transport2d_varbeta_{n}x{n}"
                                               "_p4_cn"),
                     "hbm_view": {"achieved_gbs": alg_bytes / (avg_ms * 1e-3) / 1e9,
                                  "peak_gbs": hbm, "frac": alg_bytes / (avg_ms * 1e-3) / 1e9 / hbm,
                                  "peak_source": peak_src}},
        "kernel_time_share": kernel_shares(stats),
        "mixed_precision": mixed,
        "gpu_launches": int(sum(v[0] for v in launch_counts.values())),
    }
    if standalone:
        g_pin = torch.from_numpy(g_h).pin_memory()
        u0_pin = torch.from_numpy(u0_h).pin_memory()
        u_pin = torch.empty(solver.state_shape, dtype=torch.float64).pin_memory()
        uh_pin = torch.empty(solver.trace_shape, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it_e2e = 0
        for _ in range(reps):
            solver.set_boundary(g_pin)
            solver.set_state(u0_pin)
            it_e2e += sum(solver.run(wl.n_steps))
            solver.get_state(u_pin, uh_pin)
        torch.cuda.synchronize()
        e_s = time.perf_counter() - t0
        _, _, e2e_value = combine_ranks(e_s * 1e3, trace_dof * it_e2e, ws, dev)
        out["e2e"] = {"value": e2e_value, "unit": UNIT,
                      "h2d_bytes_per_step": int(u0_h.nbytes + g_h.nbytes),
                      "d2h_bytes_per_step": int(u_pin.numel() * 8 + uh_pin.numel() * 8)}
        out["avg_sweep_ms"] = avg_ms
        out["flops_per_sweep"] = flops
    solver.close()
    return out


def fp64_sweep(info):
    """(kernel, FP64 flops one sweep executes, flops of the dense form
    2 rows NQFS) of a transport context's DFMA sweep. The sum-factorised
    sweep (hexahedra, shared operator) executes per element two 1D passes per
    face (2 NQFS q FMAs), the face scaling (NQFS) and the dense rows x NB
    product over the NB = (p+1)^3 - (p-1)^3 boundary nodes."""
    nel, nq, rows = info["n_elem"], 2 * info["dim"] * info["Nqf"], info["sweep_rows"]
    dense = 2.0 * rows * nq
    if not info.get("sum_factorised"):
        return "k_sweep_fused", dense, dense
    q = info["q"]
    nb = q ** 3 - (q - 2) ** 3
    fma = nel * (2 * nq * q + nq) + rows * nb
    return "k_sweep_sf", 2.0 * fma, dense


# the dominant kernel of each kind the profiling run times, per path
def _kernel_name(kind, precision, emulated_outer, info=None):
    emulated = precision == "fp64_emulated" or emulated_outer
    fp64_name = fp64_sweep(info)[0] if info else "k_sweep_fused"
    return {"elem": "k_ozaki (sweep mode)" if emulated else fp64_name,
            "corr": "k_sweep_tc", "step": "k_step" + (" + k_ozaki (step mode)" if emulated else ""),
            "final": "k_final" + (" / k_ozaki (reconstruction mode)" if emulated else ""),
            "face": "k_face / k_tangent", "aux": "transposes, resets, FP64 update",
            }.get(kind, kind)


def dominant_roofline(stats, info, precision, emulated_outer, fp64_peak_tf, fp64_src, peaks,
                      peak_src):
    """Roofline of the kind with the largest share of a profiled run:
    FP64 sweep on the DFMA pipe (alu), FP64-accurate sweep on the BF16 tensor
    pipe (tensor, executed digit MMAs), correction sweep (hbm)."""
    kind = max(stats, key=lambda k: stats[k][1])
    nel, nq, rows = info["n_elem"], 2 * info["dim"] * info["Nqf"], info["sweep_rows"]
    share = kernel_shares(stats).get(kind, 0.0)
    launches, ms = stats[kind]
    name = _kernel_name(kind, precision, emulated_outer, info)
    out = {"kernel": name, "kind": kind, "share": share, "launches": int(launches)}
    if kind == "elem" and name in ("k_sweep_fused", "k_sweep_sf"):
        _, flops, dense = fp64_sweep(info)
        t = ms / launches * 1e-3
        out.update({"bound": "alu", "achieved": flops / t / 1e12, "peak": fp64_peak_tf,
                    "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp64_peak_tf,
                    "peak_source": fp64_src, "flops_per_launch": flops,
                    "dense_form_equivalent_tflops": dense / t / 1e12,
                    "avg_launch_us": t * 1e6})
    elif kind == "elem":
        # digit products: 34 (i, l) pairs with i + l <= 7 of M = 128 elements,
        # N = LS (sweep rows padded to 16, then to 32), K = KP (NQFS padded to 16)
        per_row = rows // nel
        LS = ((max(16, (per_row + 15) // 16 * 16) + 31) // 32) * 32
        KP = max(16, (nq + 15) // 16 * 16)
        tiles = (nel + 127) // 128
        flops = 2.0 * 34 * 128 * LS * KP * tiles
        t = ms / launches * 1e-3
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
        out.update({"bound": "tensor", "achieved": flops / t / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak,
                    "peak_source": f"bf16_tflops_sustained of MEASURED_PEAKS.json ({peak_src})",
                    "flops_per_launch": flops, "avg_launch_us": t * 1e6,
                    "fp64_equivalent_tflops": 2.0 * rows * nq / t / 1e12,
                    "fp64_equivalent_frac_of_fp64_peak": 2.0 * rows * nq / t / 1e12 / fp64_peak_tf})
    elif kind == "corr":
        # per element: the correction at its NQFS face points (each point is
        # shared by the two elements of its face), R and the new correction at
        # its owned rows, its face ids; FP32
        bytes_ = nel * (4 * nq // 2 + 4 * 2 * (rows // nel) + 4 * 2 * info["dim"])
        t = ms / launches * 1e-3
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        out.update({"bound": "hbm", "achieved": bytes_ / t / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": bytes_ / t / 1e9 / hbm, "peak_source": peak_src,
                    "alg_bytes_per_launch": bytes_, "avg_launch_us": t * 1e6})
    return out


def run_headline(args):
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
    stream = torch.cuda.current_stream()
    n = args.n or 64
    wl = workload_3d(n, args.time_steps or 20)
    mesh = ehdg.ehdg_mesh_structured((n, n, n))

    def make(precision, tol, emulated_outer=False, inner_sweeps=None):
        return ehdg.Solver(mesh, wl.p, scheme=wl.scheme, dt=wl.dt, tol=tol, max_iter=400,
                           beta_const=wl.beta_const, precision=precision,
                           inner_sweeps=inner_sweeps or args.inner_sweeps,
                           emulated_outer=emulated_outer, stream=stream)

    t_setup0 = time.perf_counter()
    solver = make("fp64", wl.tol)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup0
    info = solver.info
    X, XF = solver.node_coords(), solver.face_point_coords()
    u0_h = np.ascontiguousarray(wl.initial(X))
    gs_h = [np.ascontiguousarray(wl.boundary(XF, k * wl.dt)) for k in range(wl.n_steps + 1)]
    u0_d = torch.from_numpy(u0_h).to(dev)
    gs_d = [torch.from_numpy(g).to(dev) for g in gs_h]
    trace_dof = info["n_face"] * info["Nqf"]

    def runner(s):
        # graph-launched steps; each step takes its inflow data first
        def one_run():
            s.set_boundary(gs_d[0])
            s.set_state(u0_d)
            its = 0
            for k in range(wl.n_steps):
                s.set_boundary(gs_d[k + 1])
                its += s.run(1)[0]
            return its
        return one_run

    one_run = runner(solver)
    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    solver.set_profiling(False)          # resets the launch counters
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters_total = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            iters_total += one_run()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launch_counts = solver.kernel_stats()
    t_max, _, value = combine_ranks(ms, trace_dof * iters_total, ws, dev)
    clocks = clk.summary()
    u_head, _ = solver.get_state()

    # end to end through host buffers (right after the device-resident
    # timing, on the same context): the initial state and every step's
    # boundary data in pinned host memory, state and trace read back
    g_pin = [torch.from_numpy(g).pin_memory() for g in gs_h]
    u0_pin = torch.from_numpy(u0_h).pin_memory()
    u_pin = torch.empty(solver.state_shape, dtype=torch.float64).pin_memory()
    uh_pin = torch.empty(solver.trace_shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_e2e = 0
    for _ in range(args.steps):
        solver.set_boundary(g_pin[0])
        solver.set_state(u0_pin)
        for k in range(wl.n_steps):
            solver.set_boundary(g_pin[k + 1])
            it_e2e += solver.run(1)[0]
        solver.get_state(u_pin, uh_pin)
    torch.cuda.synchronize()
    e_s = time.perf_counter() - t0
    _, _, e2e_value = combine_ranks(e_s * 1e3, trace_dof * it_e2e, ws, dev)
    # the library reads a boundary-data array only at the boundary faces (the
    # pinned host array through its device mapping): those bytes cross
    n_bface = int(np.count_nonzero(np.asarray(mesh["face_elem"]).reshape(-1, 2)[:, 1] < 0))
    h2d = int(u0_h.nbytes + len(gs_h) * n_bface * info["Nqf"] * 8)
    d2h = int(u_pin.numel() * 8 + uh_pin.numel() * 8)

    # per-kernel device time: the same run, every launch bracketed by CUDA
    # events on the library's stream (host-driven loop, same kernels)
    solver.set_profiling(True)
    prof_sweeps = one_run()
    stats = solver.kernel_stats()
    solver.set_profiling(False)

    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_tf, peak_txt, probe_tf, derived_tf, sms = fp64_peak(ehdg, stream, clocks.get("sm_mhz"))
    nq, rows, nel = 2 * info["dim"] * info["Nqf"], info["sweep_rows"], info["n_elem"]
    n_sweep, sweep_ms = stats["elem"]
    avg_ms = sweep_ms / max(n_sweep, 1)
    sweep_kernel, flops, dense_flops = fp64_sweep(info)
    alg_bytes = ALG_BYTES_PER_ELEM_3D * nel
    # bytes the fused sweep must move: the trace at the element's NQFS points
    # (each shared by the two elements of its face), Gy at its rows, the new
    # trace at its owned rows, its face ids
    own_bytes = nel * (8 * nq // 2 + 8 * 2 * (rows // nel) + 4 * 2 * info["dim"])
    roofline = {
        "kernel": sweep_kernel, "bound": "alu",
        "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
        "frac": flops / (avg_ms * 1e-3) / 1e12 / peak_tf, "peak_source": peak_txt,
        "fp64_probe_tflops": probe_tf, "fp64_derived_tflops": derived_tf, "sms": sms,
        "traffic": kernel_traffic(f"{sweep_kernel}@transport3d_{n}x{n}x{n}_p3_be"),
        "flops_per_sweep": flops, "dense_form_flops_per_sweep": dense_flops,
        "dense_form_equivalent_tflops": dense_flops / (avg_ms * 1e-3) / 1e12,
        "avg_sweep_us": avg_ms * 1e3, "sweeps": int(n_sweep),
        "hbm_view": {"alg_bytes_per_sweep": alg_bytes,
                     "alg_bytes_definition": "8 (n + 2 T_own) per element, n = 64, T_own = 48",
                     "achieved_gbs": alg_bytes / (avg_ms * 1e-3) / 1e9, "peak_gbs": hbm,
                     "frac": alg_bytes / (avg_ms * 1e-3) / 1e9 / hbm,
                     "peak_source": peak_src, "own_alg_bytes_per_sweep": own_bytes}}

    # the FP64 fixed point: the same run with every step converged to 1e-13
    fix = make("fp64", 1e-13)
    runner(fix)()
    u_fix, uh_fix = fix.get_state()
    fix.close()

    # time to the matched tolerance, every path
    ttt = None
    if not args.no_mixed:
        reps = max(1, min(args.steps, 3))
        ttt = {"rule": (f"every path stops when the FP64 trace residual "
                        f"||uhat^(k+1) - uhat^k||_L2(E_h) < {TOL_MATCHED_3D:g} (mixed precision: "
                        "the residual of its outer FP64 sweeps), the largest tolerance of "
                        "1e-11, 3e-12, 1e-12 at which the FP64 path lands within "
                        f"{ACCURACY_TARGET:g} relative L2 of its fixed point; the fixed point "
                        "is the FP64 path with every step converged to 1e-13"),
               "tol": TOL_MATCHED_3D, "accuracy_target": ACCURACY_TARGET,
               "timing": f"median of {reps} runs, each timed with CUDA events (runs_ms); mixed "
                         "precision keeps the inner sweep count m whose one timed run (after a "
                         "warm-up run) is fastest: m = 8, 12, 16, 20, 24, then steps of one "
                         "from the best while faster (at most 4 more)",
               "fp64_at_config_tol": {"tol": wl.tol, "ms_per_run": t_max / args.steps,
                                      "rel_l2_vs_fp64_fixed_point": rel_l2(u_head, u_fix)}}
        entries = [("fp64", "fp64", False), ("fp64_emulated", "fp64_emulated", False),
                   ("tf32", "tf32", False), ("bf16", "bf16", False),
                   ("tf32+emulated_outer", "tf32", True), ("bf16+emulated_outer", "bf16", True)]
        for name, prec, eo in entries:
            # mixed precision: the inner sweep count m that gives the fastest
            # whole run (each candidate timed over one run after a warm-up run)
            def build_m(m, prec=prec, eo=eo):
                sc = make(prec, TOL_MATCHED_3D, eo, m)
                return sc, runner(sc)
            if prec in ("tf32", "bf16") and args.tune_inner:
                s, run_s, m_kept, tried = fastest_m(INNER_GRID_3D, build_m, stream,
                                                    refine=INNER_REFINE)
            else:
                s, run_s = build_m(None)
                run_s()                                     # warm-up (captures the graph)
                m_kept, tried = None, {}
            runs_ms, its = events_ms_each(stream, run_s, reps)
            ems = statistics.median(runs_ms)      # one slow run (host jitter) does not move it
            u, uh = s.get_state()
            s.set_profiling(True)
            run_s()
            st = s.kernel_stats()
            s.set_profiling(False)
            ent = {"ms_per_run": ems, "runs_ms": [round(t, 2) for t in runs_ms],
                   "fp64_sweeps_per_run": its,
                   "rel_l2_vs_fp64_fixed_point": rel_l2(u, u_fix),
                   "rel_l2_trace_vs_fp64_fixed_point": rel_l2(uh, uh_fix),
                   "kernel_time_share": kernel_shares(st),
                   "dominant_kernel": dominant_roofline(st, s.info, prec, eo, peak_tf, peak_txt,
                                                        peaks, peak_src)}
            if prec in ("tf32", "bf16"):
                ent["inner_sweeps"] = m_kept or args.inner_sweeps
                if tried:
                    ent["inner_sweeps_tried_ms_per_run"] = tried
                ent["correction_sweeps_per_run"] = int(st.get("corr", (0, 0))[0] // 1)
            ttt[name] = ent
            s.close()
        for name, _, _ in entries:
            ttt[name]["speedup_vs_fp64"] = ttt["fp64"]["ms_per_run"] / ttt[name]["ms_per_run"]

    solver.close()
    del gs_d, g_pin

    secondary = None
    if not args.no_secondary:
        a2 = argparse.Namespace(**vars(args))
        a2.n, a2.time_steps = 0, 0
        secondary = run_2d(a2, ws, dev, stream)

    sw = None
    if not args.no_sw:
        sw = sw_variants(args)

    batch = None
    if not args.no_batch:
        # the batched mix (256 instances), at its matched-accuracy tolerance:
        # the batched loop and the autotuned schedule, FP64 and mixed
        bout, binfo = batch_variants(args, ["fp64", "fp32", "tf32", "fp64+persistent",
                                            "fp32+persistent", "fp64+tuned", "fp32+tuned",
                                            "tf32+tuned"], TOL_MATCHED_BATCH)
        batch = {"metric": "instances/s (one graph launch per step)", "config": binfo,
                 "results": bout}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"transport3d_{n}x{n}x{n}_p3_be", "n_elem": nel, "p": wl.p,
                       "beta": [float(v) for v in wl.beta_const], "scheme": "backward Euler",
                       "dt": wl.dt, "time_steps_per_run": wl.n_steps, "tol": wl.tol,
                       "trace_dof": trace_dof,
                       "trace_dof_definition": "n_face x Nqf, Nqf = (p+1)^2 face Gauss points "
                                               "(= face nodes for a constant velocity)",
                       "ms_per_step_means": "one 20-step run from the initial condition",
                       "ms_per_implicit_step": t_max / args.steps / wl.n_steps,
                       "iterations_per_run": iters_total / args.steps,
                       "rel_l2_vs_fp64_fixed_point": rel_l2(u_head, u_fix),
                       "l2": f"inputs larger than L2 ({info['device_bytes'] / 1e9:.2f} GB "
                             "resident per context; trace arrays 102 MB each)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "setup_s": round(setup_s, 3)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "h2d_definition": "initial state, plus every step's boundary data at the "
                                      f"{n_bface} boundary faces (the arrays passed are "
                                      "[n_face][Nqf]; interior entries are not read)"},
            "gpu_launches": int(sum(v[0] for v in launch_counts.values())),
            "roofline": roofline,
            "kernel_time_share": kernel_shares(stats),
            "time_to_tol": ttt,
            "secondary": secondary,
            "shallow_water": sw,
            "batch": batch,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline("3d")
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_2d_line(args):
    """--workload transport2d_varbeta: that workload's line alone."""
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
    stream = torch.cuda.current_stream()
    with ClockSampler(local) as clk:
        res = run_2d(args, ws, dev, stream, standalone=True)
    clocks = clk.summary()
    peak_tf, peak_txt, probe_tf, derived_tf, sms = fp64_peak(ehdg, stream, clocks.get("sm_mhz"))
    r = res["roofline"]
    r.update({"achieved": r["achieved_tflops"], "peak": peak_tf, "unit": "TFLOP/s",
              "frac": r["achieved_tflops"] / peak_tf, "peak_source": peak_txt})
    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_run"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {k: res[k] for k in ("workload", "n_elem", "p", "time_steps_per_run",
                                               "dt", "tol", "trace_dof", "trace_dof_definition",
                                               "iterations_per_run", "setup_s")},
                "e2e": res["e2e"], "gpu_launches": res["gpu_launches"], "roofline": r,
                "kernel_time_share": res["kernel_time_share"],
                "mixed_precision": res["mixed_precision"], "clocks": clocks}
        line["config"]["l2"] = "inputs larger than L2 (per-element operators resident)"
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline("2d")
        print(json.dumps(line), flush=True)
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
    n = args.n or {"transport3d": 64, "sw2d": 512, "steady2d": 256}.get(args.workload, 16)
    n_steps = args.time_steps or {"transport3d": 20, "sw2d": 20}.get(args.workload, 10)
    dt_note = None
    if args.workload == "transport3d":
        wl = W.transport_3d(n=(n, n, n), p=3, n_steps=n_steps)
        precisions = ["fp64", "fp64+tiles", "fp64_emulated", "tf32", "bf16", "fp32",
                      "bf16+emulated_outer"]
    elif args.workload == "sw2d":
        # dt at which Theorem 2 holds on this mesh: h / (dt (p+1)(p+2)) = 3.9, C = 0.34
        wl = W.sw_2d(n=(n, n), p=3, dt=2.5e-5, n_steps=n_steps)
        dt_note = SW_DT_NOTE.replace("and 20 steps (not 100)",
                                     f"and {n_steps} steps (not 100)")
        precisions = ["fp64", "fp64_emulated", "tf32", "bf16", "fp32", "bf16+emulated_outer"]
    elif args.workload == "steady2d":
        # the steady solve of Sec. 4.1 (one "step", many iterations)
        wl = W.steady_2d_smooth(n=(n, n), p=4)
        precisions = ["fp64", "fp32", "bf16"]
    else:
        wl = W.transport_2d_small(n=(n, n), p=2, n_steps=n_steps)
        precisions = ["fp64", "fp64_emulated", "tf32", "fp32"]
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
    if dt_note:
        info["dt_note"] = dt_note
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


SW_DT_NOTE = ("changed workload: dt = 2.5e-5 (not 1e-3) and 20 steps (not 100), because at "
              "dt = 1e-3 on this mesh h / (dt (p+1)(p+2)) = 0.098 < 1, Theorem 2's "
              "contraction condition fails and the eHDG iteration grows by dt (p+1)(p+2) / h "
              "per iteration (pinned on the oracle); at 2.5e-5 the ratio is 3.9 and C = 0.34")


def sw_variants(args):
    """Config 3: linearised shallow water (Phi = 1, walls) on 512^2 quads, p = 3,
    one shared 48 x 48 local operator, backward Euler dt = 2.5e-5 x 20 steps.
    The FP64 fixed point is the FP64 run with every step converged to 1e-13;
    the stopping tolerance is the largest of 1e-10, 1e-11, 3e-12, 1e-12 at which
    the FP64 run lands within 1e-10 relative L2 of it (chosen in the run), and
    every path (FP64 on the DFMA pipe, FP64-accurate on the BF16 tensor cores,
    TF32/BF16 tensor-core corrections with FP64 defect correction, with DFMA or
    tensor-core outer sweeps) stops at that tolerance."""
    import torch
    from paper_1601_06681_gb300 import ehdg
    from paper_1601_06681_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    wl = W.sw_2d(n=(512, 512), p=3, dt=2.5e-5, n_steps=20)
    mesh = ehdg.ehdg_mesh_structured(wl.n, boundary_tag=2)

    def make(prec, tol, max_iter=400, inner_sweeps=None):
        base, _, opt = prec.partition("+")
        return ehdg.Solver(mesh, wl.p, pde="sw", scheme=wl.scheme, dt=wl.dt, tol=tol,
                           max_iter=max_iter, precision=base,
                           inner_sweeps=inner_sweeps or args.inner_sweeps, stream=stream,
                           emulated_outer=(opt == "emulated_outer"), Phi=wl.Phi)

    s = make("fp64", 1e-13, 4000)
    X, XF = s.node_coords(), s.face_point_coords()
    u0 = torch.from_numpy(np.ascontiguousarray(wl.initial(X))).cuda()
    g0 = torch.from_numpy(np.ascontiguousarray(wl.boundary(XF, 0.0))).cuda()

    def run(sol):
        sol.set_boundary(g0)
        sol.set_state(u0)
        return sum(sol.run(wl.n_steps))

    run(s)
    u_fix = s.get_state()[0]
    s.close()
    tol, tol_errs = 1e-12, {}
    for t in (1e-10, 1e-11, 3e-12, 1e-12):
        s = make("fp64", t)
        run(s)
        tol_errs[f"{t:g}"] = rel_l2(s.get_state()[0], u_fix)
        s.close()
        if tol_errs[f"{t:g}"] <= ACCURACY_TARGET:
            tol = t
            break
    reps = max(1, min(args.steps, 5))
    out = {}
    for prec in ["fp64", "fp64_emulated", "tf32", "bf16", "tf32+emulated_outer",
                 "bf16+emulated_outer"]:
        base = prec.partition("+")[0]
        m, tried = None, {}
        if base in ("tf32", "bf16") and args.tune_inner:
            # the inner sweep count whose whole run is fastest
            def build(mm, prec=prec):
                c = make(prec, tol, inner_sweeps=mm)
                return c, (lambda: run(c))
            s, _, m, tried = fastest_m((2, 3, 4, 6, 8, 12), build, stream, refine=INNER_REFINE)
        else:
            s = make(prec, tol)
        run(s)                                        # warm-up (captures the graphs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = 0
        for _ in range(reps):
            its = run(s)
        e1.record(stream)
        torch.cuda.synchronize()
        ent = {"ms_per_run": e0.elapsed_time(e1) / reps, "fp64_sweeps_per_run": int(its),
               "rel_l2_vs_fp64_fixed_point": rel_l2(s.get_state()[0], u_fix)}
        if base in ("tf32", "bf16"):
            ent["inner_sweeps"] = m if m is not None else args.inner_sweeps
            if tried:
                ent["inner_sweeps_tried_ms_per_run"] = tried
        out[prec] = ent
        s.close()
    for prec in out:
        out[prec]["speedup_vs_fp64"] = out["fp64"]["ms_per_run"] / out[prec]["ms_per_run"]
    info = {"workload": wl.name, "n_elem": int(np.prod(wl.n)), "p": wl.p, "fields": 3,
            "local_operator": "one shared 48 x 48", "dt": wl.dt, "time_steps": wl.n_steps,
            "dt_note": SW_DT_NOTE, "tol": tol,
            "tol_rule": "the largest of 1e-10, 1e-11, 3e-12, 1e-12 at which FP64 lands within "
                        "1e-10 relative L2 of its fixed point (every step to 1e-13)",
            "fp64_rel_l2_vs_fixed_point_by_tol": tol_errs, "runs_timed": reps,
            "inner_sweeps_rule": "mixed precision keeps the m whose whole run is fastest (one "
                                 "timed run after a warm-up run each): m = 2, 3, 4, 6, 8, 12, "
                                 "then steps of one from the best while faster (at most 4 more)"}
    return {"metric": "time-to-tol per run, mixed vs FP64", "config": info, "results": out}


# stopping tolerance of the batched mix (config 5) at matched accuracy: the
# largest of 1e-11, 3e-12, 1e-12 at which every instance's FP64 state lies
# within 1e-10 relative L2 of its fixed point (at 1e-11: 21 of 256 above)
TOL_MATCHED_BATCH = 3e-12


def batch_variants(args, variants, tol, profile_loop=True):
    """Config 5: independent 2D transport instances (N 8..128, p 1..5) stepped
    together, one graph launch per time step, every instance to `tol`.
    Variant "prec" iterates in the batched loop (one launch per kernel and
    iteration over every unconverged instance); "prec+branches" runs every
    instance's own loop on the graph's branches; "prec+persistent" the
    loop's persistent form (every iteration of a step in one launch, FP64 and
    FP32 corrections); "prec+tuned" takes the schedule from
    ehdg_batch_autotune_schedule (loop, persistent, or branches with 16/32/64
    of them); "+inner" tunes the inner sweep count m; "+tiles" the
    fused FP64 sweep's tile. Branch counts come from the batch autotuners,
    timed over the same run after a warm-up run (setup, outside the timed
    run). Every variant's final states are compared with the instances' FP64
    fixed points (every step converged to 1e-13)."""
    import torch
    from paper_1601_06681_gb300 import ehdg
    from paper_1601_06681_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    wls = W.batched_mix(n_inst=args.n_inst)

    def make_specs(base, opt, tol_i, max_iter=400):
        specs = []
        for wl in wls:
            mesh = ehdg.ehdg_mesh_structured(wl.n)
            specs.append(dict(mesh=mesh, p=wl.p, scheme=wl.scheme, dt=wl.dt, tol=tol_i,
                              max_iter=max_iter, beta_const=wl.beta_const, precision=base,
                              inner_sweeps=args.inner_sweeps,
                              emulated_outer=(opt == "emulated_outer")))
        return specs

    def start(b):
        ins = []
        for wl, s in zip(wls, b.instances):
            X, XF = s.node_coords(), s.face_point_coords()
            s.set_boundary(wl.u0_fn(XF))
            ins.append(torch.from_numpy(np.ascontiguousarray(wl.initial(X))).cuda())
        return ins

    bfix = ehdg.Batch(make_specs("fp64", "", 1e-13, max_iter=4000), stream=stream)
    for s, u0 in zip(bfix.instances, start(bfix)):
        s.set_state(u0)
    bfix.run(wls[0].n_steps)
    u_fix = [s.get_state()[0] for s in bfix.instances]
    bfix.close()

    def accuracy(b):
        errs = np.array([rel_l2(s.get_state()[0], uf) for s, uf in zip(b.instances, u_fix)])
        return {"max": float(errs.max()), "median": float(np.median(errs)),
                "instances_above_target": int((errs > ACCURACY_TARGET).sum())}

    out = {}
    for prec in variants:
        base, _, opt = prec.partition("+")
        t0 = time.perf_counter()
        b = ehdg.Batch(make_specs(base, opt, tol), stream=stream)
        if opt == "branches":
            b.set_loop(False)
        elif opt == "persistent":
            b.set_loop("persistent")
        setup = time.perf_counter() - t0
        inputs = start(b)

        def reset():
            for s, u0 in zip(b.instances, inputs):
                s.set_state(u0)

        def one_run():
            reset()
            return b.run(wls[0].n_steps)

        one_run()                                     # warm-up (captures the graph)
        reset()
        tuned = {}
        if opt == "tiles":
            tuned["tile_ft"], _ = b.autotune_sweep_tile()
        if opt == "inner":
            tuned["inner_sweeps"], _ = b.autotune_inner_sweeps((4, 6, 8, 12))
        if args.batch_chains > 0:
            b.set_chains(args.batch_chains)
            chains = args.batch_chains
        else:
            chains, _ = b.autotune_chains()
        if opt == "tuned":
            mode, chains, _ = b.autotune_schedule((16, 32, 64))
            tuned["schedule"] = ("branches", "loop", "persistent")[mode]
        one_run()                                     # recapture with the tuned settings
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iters, times = one_run()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[prec] = {"instances_per_s": len(wls) / wall, "wall_s": wall, "setup_s": setup,
                     "p50_instance_ms": float(np.percentile(times, 50) * 1e3),
                     "p99_instance_ms": float(np.percentile(times, 99) * 1e3),
                     "sweeps_total": int(iters.sum()), "chains": chains,
                     "rel_l2_vs_fp64_fixed_point": accuracy(b), **tuned}
        if (profile_loop and opt not in ("branches", "tuned", "emulated_outer")
                and base in ("fp64", "fp32", "tf32", "bf16")):
            # kernel accounting of the batched loop: the same run with its
            # steps driven from the host and every launch timed
            b.set_profiling(True)
            one_run()
            st = b.kernel_stats()
            b.set_profiling(False)
            out[prec]["loop_kernel_ms"] = {k: round(v[1], 3) for k, v in st.items() if v[0]}
            out[prec]["loop_kernel_launches"] = {k: v[0] for k, v in st.items() if v[0]}
        b.close()
    ref = out.get("fp64+tuned", out.get("fp64"))
    if ref:
        for prec in variants:
            out[prec]["speedup_vs_fp64"] = ref["wall_s"] / out[prec]["wall_s"]
    info = {"workload": f"batched_mix_{args.n_inst}", "time_steps": wls[0].n_steps,
            "dt": wls[0].dt, "tol": tol,
            "tol_reading": "the largest of 1e-11, 3e-12, 1e-12 at which every instance's FP64 "
                           "state lies within 1e-10 of its fixed point (the mix's own 1e-10 "
                           "leaves FP64 up to 2.4e-9 away)" if tol == TOL_MATCHED_BATCH else
                           "given on the command line",
            "accuracy": "relative L2 of each instance's final volume state from its FP64 "
                        "fixed point (every step converged to 1e-13): max and median over "
                        f"instances, and how many exceed {ACCURACY_TARGET:g}",
            "elements_total": int(sum(np.prod(w.n) for w in wls)),
            "per_instance_time": "device time from the instance's step start to its "
                                 "convergence (batched loop) or to its last kernel "
                                 "(branches), summed over the steps",
            "speedup_reference": "fp64+tuned" if "fp64+tuned" in out else "fp64"}
    return out, info


def batch_workload(args):
    """The batch workload alone: every variant, one JSON line."""
    import torch
    from paper_1601_06681_gb300 import build, ehdg
    torch.cuda.set_device(0)
    build.build()
    ehdg.load()
    variants = ["fp64", "fp32", "tf32", "bf16", "fp64+persistent", "fp32+persistent",
                "fp64+branches", "fp32+branches", "tf32+branches", "fp64+tuned", "fp32+tuned",
                "tf32+tuned", "fp32+inner", "tf32+inner", "fp64_emulated",
                "tf32+emulated_outer"]
    if args.batch_variants:
        variants = [v for v in args.batch_variants.split(",") if v]
    tol = args.batch_tol if args.batch_tol > 0 else TOL_MATCHED_BATCH
    out, info = batch_variants(args, variants, tol)
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
    elif args.workload == "headline":
        run_headline(args)
    elif args.workload == "transport2d_varbeta":
        run_2d_line(args)
    else:
        compare_workload(args)


if __name__ == "__main__":
    main()
