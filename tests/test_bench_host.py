"""Host-side logic of bench.py that needs no GPU: the oracle baseline spread
over host cores (one spawned process per core)."""
import importlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    # imported by name, so that the spawned workers find the same functions
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_oracle_pool_runs_one_sample_per_process():
    bench = load_bench()
    one_3d = bench.oracle_sample_3d(n_side=2, n_time=1)[1]
    one_2d = bench.oracle_sample_2d(n_side=4, n_time=1)[1]
    pool = bench.OraclePool(cores=2)
    try:
        wall, units, sample = pool.run("3d", n_side=2, n_time=1)
        wall2, units2, sample2 = pool.run("2d", n_side=4, n_time=1)
    finally:
        pool.close()
    assert wall > 0 and wall2 > 0
    # two independent copies of the same deterministic sample
    assert units == 2 * one_3d and units2 == 2 * one_2d
    assert sample.startswith("2 processes") and "64^3" in sample and "256x256" in sample2


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        bench = load_bench()
        # rank r times (r + 1) ms and processes 100 (r + 1) units
        t_max, units, value = bench.combine_ranks(float(rank + 1), 100 * (rank + 1), ws, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{t_max} {units} {value}\n")
    finally:
        dist.destroy_process_group()


def test_combine_ranks_over_two_gloo_ranks(tmp_path):
    """The multi-rank reduction of the benchmark (replicas: max time over
    ranks, units summed) on world size 2 with the gloo backend."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for rank in range(2):
        t_max, units, value = map(float, open(tmp_path / f"rank{rank}.txt").read().split())
        assert t_max == 2.0
        assert units == 300.0
        assert value == 300.0 / 2e-3
    bench = load_bench()
    assert bench.combine_ranks(4.0, 50, 1) == (4.0, 50, 50 / 4e-3)


def test_inner_sweep_tuner_keeps_the_fastest_run_and_closes_the_rest():
    """fastest_m: every candidate is built, warmed up once and timed once; the
    fastest one's context stays open, every other is closed, and the timings
    are reported per candidate."""
    bench = load_bench()
    cost = {4: 9.0, 8: 5.0, 12: 3.0, 16: 7.0}

    class Ctx:
        def __init__(self, m):
            self.m, self.closed, self.runs = m, False, 0

        def close(self):
            self.closed = True

    built = []

    def build(m):
        c = Ctx(m)
        built.append(c)

        def run():
            c.runs += 1
            return m
        return c, run

    ctx, run, m, tried = bench.fastest_m((4, 8, 12, 16), build, None,
                                         timer=lambda r: cost[r()])
    assert m == 12 and ctx.m == 12 and not ctx.closed and run() == 12
    assert tried == {"4": 9.0, "8": 5.0, "12": 3.0, "16": 7.0}
    assert [c.closed for c in built] == [True, True, False, True]
    assert all(c.runs >= 2 for c in built)      # a warm-up run, then the timed run


def test_inner_sweep_tuner_default_timer_uses_the_event_timer(monkeypatch):
    """Without a timer, fastest_m times each candidate with events_ms_each on
    the given stream (one run)."""
    bench = load_bench()
    calls = []

    def fake_events(stream, fn, reps):
        calls.append((stream, reps))
        return [float(fn())], None

    monkeypatch.setattr(bench, "events_ms_each", fake_events)

    class Ctx:
        def close(self):
            pass

    ctx, run, m, tried = bench.fastest_m((6, 3), lambda m: (Ctx(), lambda: m), "s0")
    assert m == 3 and tried == {"6": 6.0, "3": 3.0}
    assert calls == [("s0", 1), ("s0", 1)]


def _tuner_fixture():
    class Ctx:
        def __init__(self, m):
            self.m, self.closed = m, False

        def close(self):
            self.closed = True

    built = {}

    def build(m):
        c = Ctx(m)
        built[m] = c
        return c, (lambda: m)
    return build, built


def test_inner_sweep_tuner_refines_between_grid_points():
    """With refine, the search steps by one from the fastest grid point in the
    direction that is faster and stops where the next step is slower: run time
    falls from 16 to 14 and rises at 13 (the step shape of an integer outer
    iteration count)."""
    bench = load_bench()
    cost = {8: 94.0, 12: 94.5, 13: 83.0, 14: 82.2, 15: 86.0, 16: 87.3, 17: 88.0,
            20: 97.3, 24: 107.0}
    build, built = _tuner_fixture()
    ctx, run, m, tried = bench.fastest_m((8, 12, 16, 20, 24), build, None,
                                         timer=lambda r: cost[r()], refine=4)
    assert m == 14 and ctx.m == 14 and not ctx.closed and run() == 14
    assert list(tried) == ["8", "12", "16", "20", "24", "15", "14", "13"]
    assert [k for k, c in built.items() if not c.closed] == [14]


def test_inner_sweep_tuner_refine_is_bounded_and_stays_in_range():
    """The refine steps build at most `refine` more contexts, never leave the
    library's range 1..64 and never rebuild a tried count; refine = 0 (the
    default) tries the grid alone."""
    bench = load_bench()
    build, built = _tuner_fixture()
    ctx, _, m, tried = bench.fastest_m((4, 8), build, None, timer=lambda r: float(r()),
                                       refine=2)
    assert (m, list(tried)) == (2, ["4", "8", "3", "2"])       # downhill, 2 steps only
    build, built = _tuner_fixture()
    ctx, _, m, tried = bench.fastest_m((2, 1), build, None, timer=lambda r: float(r()),
                                       refine=4)
    assert (m, list(tried)) == (1, ["2", "1"])                 # m = 0 is out of range
    build, built = _tuner_fixture()
    ctx, _, m, tried = bench.fastest_m((64, 60), build, None, timer=lambda r: -float(r()),
                                       refine=4)
    assert (m, list(tried)) == (64, ["64", "60", "63"])        # 65 is out of range
    build, built = _tuner_fixture()
    ctx, _, m, tried = bench.fastest_m((4, 8), build, None, timer=lambda r: float(r()))
    assert (m, list(tried)) == (4, ["4", "8"])


def _bench_cmd(args, env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_line_on_the_gpu_arms_workload_and_metric():
    """bench.py --impl reference (the oracle on the host cores, no GPU): one
    JSON line with the GPU arm's metric, unit, direction and workload name, a
    cpu_baseline describing the run and an e2e with no host-device bytes."""
    bench = load_bench()
    out = _bench_cmd(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                     {"WORLD_SIZE": "1", "RANK": "0"})
    assert len(out) == 1
    d = out[0]
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["higher_is_better"]) == (bench.METRIC, bench.UNIT, True)
    assert d["config"]["workload"] == "transport3d_64x64x64_p3_be"
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs and prints the reference line."""
    assert _bench_cmd(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                      {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == []


def test_traffic_record_is_dropped_once_the_kernel_source_changes(tmp_path, monkeypatch):
    """kernel_traffic returns the recorded DRAM bytes only while the kernel's
    source files hash to the value stored with the capture; an edit to any of
    them makes the bench report no traffic (null) instead of a stale figure."""
    import json
    bench = load_bench()
    csrc = tmp_path / "paper_1601_06681_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "a.cu").write_text("kernel a\n")
    (csrc / "b.cuh").write_text("helper b\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"k_a@w": {"bytes_per_sweep": 1234, "sources": ["a.cu", "b.cuh"],
                     "source_sha": bench.source_sha(["a.cu", "b.cuh"])}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.kernel_traffic("k_a@w") == 1234
    assert bench.kernel_traffic("k_other@w") is None
    (csrc / "b.cuh").write_text("helper b, changed\n")
    assert bench.kernel_traffic("k_a@w") is None


def test_committed_traffic_records_name_existing_sources():
    """Every committed traffic record names source files that exist, with the
    ncu command that measured it."""
    import json
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        recs = json.load(fh)
    assert recs
    for key, ent in recs.items():
        assert "@" in key and ent["bytes_per_sweep"] > 0
        assert "--clock-control none" in ent["command"]
        for s in ent["sources"]:
            assert os.path.exists(os.path.join(ROOT, "paper_1601_06681_gb300", "csrc", s)), s


def test_clock_summary_reports_median_clock_and_every_active_throttle_reason():
    """ClockSampler.summary over nvidia-smi's CSV (no units, no header): the
    median SM clock, the maximum clock and each throttle reason seen Active in
    any sample; lines it cannot parse are skipped; no sample at all is
    reported as unsampled rather than as a clean run."""
    bench = load_bench()
    cs = bench.ClockSampler(0)
    cs.out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ])
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0,
                 "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    cs.out = ""
    assert cs.summary()["reasons"] == ["unsampled"]


def test_measured_peaks_are_read_from_the_committed_file():
    """The roofline denominators come from MEASURED_PEAKS.json when it exists
    (labelled measured), else the stated fallback figures."""
    import json
    bench = load_bench()
    peaks, src = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            assert (peaks, src) == (json.load(fh), "measured")
        assert peaks["hbm_gbs"] > 0
    else:
        assert src == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_fp64_sweep_flops_match_the_per_element_counts():
    """The roofline's FP64 work per sweep of the 64^3, p = 3 headline: the
    sum-factorised sweep executes 2 x 96 x 4 (two 1D passes over the 96 face
    points) + 96 (face scaling) + 48 x 56 (owned rows x boundary nodes) =
    3,552 FMAs per element; the dense form it replaces 48 x 96 = 4,608."""
    bench = load_bench()
    nel = 64 ** 3
    info = {"n_elem": nel, "dim": 3, "Nqf": 16, "q": 4, "sweep_rows": 48 * nel,
            "sum_factorised": 1}
    name, flops, dense = bench.fp64_sweep(info)
    assert name == "k_sweep_sf"
    assert flops == 2.0 * 3552 * nel == 1862270976.0
    assert dense == 2.0 * 4608 * nel
    name, flops, dense = bench.fp64_sweep(dict(info, sum_factorised=0))
    assert name == "k_sweep_fused" and flops == dense == 2.0 * 4608 * nel
