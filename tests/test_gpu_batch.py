"""Batched form: independent instances stepped by one CUDA graph launch per
time step give the same results as solo runs (and as the oracle)."""
import zlib

import numpy as np
import pytest

from oracle.ehdg import Problem
from oracle.geometry import face_point_coords, node_coords
from paper_1601_06681_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ehdg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_06681_gb300 import build, ehdg as E
    build.build()
    E.load()
    return E


def instances(n=12, seed=77):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx, ny = int(rng.integers(3, 13)), int(rng.integers(3, 13))
        p = int(rng.integers(1, 5))
        th = rng.uniform(0, 2 * np.pi)
        beta = rng.uniform(0.5, 1.5) * np.array([np.cos(th), np.sin(th)])
        # the FP64-accurate tensor-core path among them: instances of different
        # shapes launch the same kernels with different shared-memory sizes
        precision = ["fp64", "tf32", "fp32", "bf16", "fp64_emulated", "tf32+emulated_outer"][i % 6]
        base, _, opt = precision.partition("+")
        mesh = W.structured_mesh((nx, ny))
        prob = Problem(mesh, p, scheme="be", dt=0.01, beta_const=beta)
        X = node_coords(mesh, p)
        XF = face_point_coords(mesh, p, prob.ref.q)
        c = rng.uniform(0.2, 0.8, 2)
        s = rng.uniform(0.05, 0.15)
        u0 = W.gaussian(X, c, s)[:, None, :]
        g = W.gaussian(XF, c, s)
        kw = dict(mesh=mesh, p=p, scheme="be", dt=0.01, tol=1e-12, max_iter=500,
                  beta_const=beta, precision=base, inner_sweeps=4,
                  emulated_outer=(opt == "emulated_outer"))
        out.append((kw, prob, u0, g))
    return out


def test_batch_matches_solo_runs_and_oracle(ehdg):
    inst = instances()
    n_steps = 3
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        iters, times = b.run(n_steps)
        batch_states = [s.get_state() for s in b.instances]
    assert np.all(times > 0)
    for i, (kw, prob, u0, g) in enumerate(inst):
        args = dict(kw)
        mesh = args.pop("mesh")
        p = args.pop("p")
        with ehdg.Solver(mesh, p, **args) as s:
            s.set_boundary(g)
            s.set_state(u0)
            solo_iters = s.run(n_steps)
            u, uh = s.get_state()
        assert list(iters[i]) == solo_iters, i
        assert np.array_equal(batch_states[i][0], u), i
        assert np.array_equal(batch_states[i][1], uh), i
        ou, _, _, _ = prob.run(u0, n_steps, g_of_t=lambda t: g, tol=1e-13, max_iter=2000)
        err = np.linalg.norm(u - ou) / np.linalg.norm(ou)
        assert err < 1e-10, (i, kw["precision"], err)


def run_batch(ehdg, inst, n_steps, chains=None, tune=None):
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        if chains is not None:
            b.set_chains(chains)
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        tuned = None
        if tune is not None:
            before = [s.get_state() for s in b.instances]
            tuned = b.autotune_chains(tune)
            after = [s.get_state() for s in b.instances]
            for (u0_, uh0_), (u1_, uh1_) in zip(before, after):
                assert np.array_equal(u0_, u1_) and np.array_equal(uh0_, uh1_)
        iters, _ = b.run(n_steps)
        return iters, [s.get_state() for s in b.instances], tuned


def test_branch_count_does_not_change_results(ehdg):
    """The graph's branch count only changes which steps run side by side:
    every instance's iterations and state are the same, bit for bit."""
    inst = instances(n=7, seed=5)
    ref_iters, ref_states, _ = run_batch(ehdg, inst, 2)
    for k in (1, 3, 7, 64):
        iters, states, _ = run_batch(ehdg, inst, 2, chains=k)
        assert np.array_equal(iters, ref_iters), k
        for (u, uh), (ru, ruh) in zip(states, ref_states):
            assert np.array_equal(u, ru) and np.array_equal(uh, ruh), k


def test_chain_autotuner_keeps_states_and_results(ehdg):
    inst = instances(n=7, seed=6)
    ref_iters, ref_states, _ = run_batch(ehdg, inst, 2)
    iters, states, (best, ms) = run_batch(ehdg, inst, 2, tune=(1, 2, 7))
    assert best in (1, 2, 7) and 0 < ms < 1e300
    assert np.array_equal(iters, ref_iters)
    for (u, uh), (ru, ruh) in zip(states, ref_states):
        assert np.array_equal(u, ru) and np.array_equal(uh, ruh)


def test_batch_tile_autotuner_keeps_states_and_results(ehdg):
    inst = instances(n=7, seed=7)
    ref_iters, ref_states, _ = run_batch(ehdg, inst, 2)
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        before = [s.get_state() for s in b.instances]
        ft, ms = b.autotune_sweep_tile((2, 8))
        assert ft in (2, 8) and 0 < ms < 1e300
        for (u0_, uh0_), s in zip(before, b.instances):
            u1_, uh1_ = s.get_state()
            assert np.array_equal(u0_, u1_) and np.array_equal(uh0_, uh1_)
        iters, _ = b.run(2)
        states = [s.get_state() for s in b.instances]
    assert np.array_equal(iters, ref_iters)
    for (u, uh), (ru, ruh) in zip(states, ref_states):
        assert np.array_equal(u, ru) and np.array_equal(uh, ruh)


def test_batch_inner_sweep_autotuner(ehdg):
    inst = instances(n=6, seed=8)            # two of each mixed precision among them
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        before = [s.get_state() for s in b.instances]
        m, ms = b.autotune_inner_sweeps((3, 6))
        assert m in (3, 6) and 0 < ms < 1e300
        for (u0_, uh0_), s in zip(before, b.instances):
            u1_, uh1_ = s.get_state()
            assert np.array_equal(u0_, u1_) and np.array_equal(uh0_, uh1_)
        b.run(2)
        states = [s.get_state() for s in b.instances]
    for (kw, prob, u0, g), (u, uh) in zip(inst, states):
        ou, _, _, _ = prob.run(u0, 2, g_of_t=lambda t: g, tol=1e-13, max_iter=2000)
        assert np.linalg.norm(u - ou) / np.linalg.norm(ou) < 1e-10, kw["precision"]
    fp64_only = [dict(kw, precision="fp64", emulated_outer=False) for kw, _, _, _ in inst[:2]]
    with ehdg.Batch(fp64_only) as b:
        with pytest.raises(ehdg.EhdgError) as ei:
            b.autotune_inner_sweeps((3, 6))
        assert ei.value.status == 1


def loop_instances(n=10, seed=31, precisions=("fp64", "tf32", "bf16")):
    """Instances the batched loop supports (2D, constant velocity, uniform
    mesh), of different sizes, degrees and precisions."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx, ny = int(rng.integers(2, 17)), int(rng.integers(2, 17))
        p = int(rng.integers(1, 6))
        th = rng.uniform(0.05, 1.5) + (np.pi / 2) * int(rng.integers(0, 4))
        beta = rng.uniform(0.5, 1.5) * np.array([np.cos(th), np.sin(th)])
        mesh = W.structured_mesh((nx, ny))
        prob = Problem(mesh, p, scheme="be", dt=0.01, beta_const=beta)
        X = node_coords(mesh, p)
        XF = face_point_coords(mesh, p, prob.ref.q)
        c = rng.uniform(0.2, 0.8, 2)
        s = rng.uniform(0.05, 0.15)
        kw = dict(mesh=mesh, p=p, scheme="be", dt=0.01, tol=1e-12, max_iter=500,
                  beta_const=beta, precision=precisions[i % len(precisions)], inner_sweeps=3 + i % 3)
        out.append((kw, prob, W.gaussian(X, c, s)[:, None, :], W.gaussian(XF, c, s)))
    return out


def run_loop(ehdg, inst, n_steps, loop=True):
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        b.set_loop(loop)
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        iters, times = b.run(n_steps)
        return iters, times, [s.get_state() for s in b.instances]


def test_batched_loop_matches_solo_runs_bitwise(ehdg):
    """Every instance iterating in the batched loop (one launch per kernel and
    iteration over all unconverged instances) gives the iterations and the
    state of its solo run, bit for bit, and the oracle's solution."""
    inst = loop_instances()
    n_steps = 3
    iters, times, states = run_loop(ehdg, inst, n_steps)
    assert np.all(times > 0)
    for i, (kw, prob, u0, g) in enumerate(inst):
        args = dict(kw)
        mesh = args.pop("mesh")
        p = args.pop("p")
        with ehdg.Solver(mesh, p, **args) as s:
            s.set_boundary(g)
            s.set_state(u0)
            solo_iters = s.run(n_steps)
            u, uh = s.get_state()
        assert list(iters[i]) == solo_iters, (i, kw["precision"])
        assert np.array_equal(states[i][0], u), (i, kw["precision"])
        assert np.array_equal(states[i][1], uh), (i, kw["precision"])
        ou, _, _, _ = prob.run(u0, n_steps, g_of_t=lambda t: g, tol=1e-13, max_iter=2000)
        assert np.linalg.norm(u - ou) / np.linalg.norm(ou) < 1e-10, (i, kw["precision"])


def test_batched_loop_equals_branch_graph(ehdg):
    """The loop on and off (every instance's own loop on the graph's branches)
    give the same iterations and states, bit for bit, also with instances
    the loop does not take (FP32 corrections, the FP64-accurate tensor-core
    path) in the same batch."""
    inst = loop_instances(n=9, seed=32, precisions=("fp64", "tf32", "bf16", "fp32",
                                                     "fp64_emulated"))
    a_iters, _, a_states = run_loop(ehdg, inst, 2, loop=True)
    b_iters, _, b_states = run_loop(ehdg, inst, 2, loop=False)
    assert np.array_equal(a_iters, b_iters)
    for (u, uh), (ru, ruh) in zip(a_states, b_states):
        assert np.array_equal(u, ru) and np.array_equal(uh, ruh)


def test_batched_loop_with_several_tiles_per_block_equals_branch_graph(ehdg):
    """Enough tensor-core correction tiles that each block of the batched
    correction sweep takes a run of several, across instances of different
    degrees (its staged operator changes inside the run): the loop and the
    branch graph (single-problem kernels) still agree bit for bit."""
    rng = np.random.default_rng(35)
    inst = []
    for i in range(28):
        n = int(rng.integers(96, 129))
        p = 1 + i % 5
        th = rng.uniform(0.05, 1.5) + (np.pi / 2) * (i % 4)
        beta = rng.uniform(0.5, 1.5) * np.array([np.cos(th), np.sin(th)])
        mesh = W.structured_mesh((n, n))
        X = node_coords(mesh, p)
        XF = face_point_coords(mesh, p, p + 1)     # Gauss points: q = p + 1 (constant velocity)
        kw = dict(mesh=mesh, p=p, scheme="be", dt=0.01, tol=1e-10, max_iter=500,
                  beta_const=beta, precision=("tf32", "bf16")[i % 2], inner_sweeps=4)
        inst.append((kw, None, W.gaussian(X, (0.4, 0.6), 0.1)[:, None, :],
                     W.gaussian(XF, (0.4, 0.6), 0.1)))
    a_iters, _, a_states = run_loop(ehdg, inst, 1, loop=True)
    b_iters, _, b_states = run_loop(ehdg, inst, 1, loop=False)
    assert np.array_equal(a_iters, b_iters)
    for (u, uh), (ru, ruh) in zip(a_states, b_states):
        assert np.array_equal(u, ru) and np.array_equal(uh, ruh)


def test_schedule_autotuner_keeps_states_and_results(ehdg):
    """The loop-or-branches autotuner restores every state and picks a
    schedule whose results equal the untuned run's bit for bit."""
    inst = loop_instances(n=8, seed=36, precisions=("fp64", "tf32", "fp32"))
    ref_iters, _, ref_states = run_loop(ehdg, inst, 2)
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        b.run(2)                                   # the run the tuner times
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_state(u0)
        before = [s.get_state() for s in b.instances]
        mode, k, ms = b.autotune_schedule((2, 4))
        assert 0 < ms < 1e300 and mode in (0, 1, 2) and (mode or k in (2, 4))
        for (u, uh), s in zip(before, b.instances):
            su, suh = s.get_state()
            assert np.array_equal(u, su) and np.array_equal(uh, suh)
        iters, _ = b.run(2)
        states = [s.get_state() for s in b.instances]
    assert np.array_equal(iters, ref_iters)
    for (u, uh), (ru, ruh) in zip(states, ref_states):
        assert np.array_equal(u, ru) and np.array_equal(uh, ruh)


@pytest.mark.parametrize("precisions", [("fp64",), ("fp64", "fp32"), ("fp32", "fp64", "tf32")])
def test_persistent_loop_matches_solo_runs_bitwise(ehdg, precisions):
    """The loop's persistent form (every iteration of a step in one launch,
    each instance through its own stages at its own pace) gives every
    instance's solo iterations and state bit for bit; with a TF32 instance in
    the batch it falls back to the loop of launches, with the same result."""
    inst = loop_instances(n=12, seed=41, precisions=precisions)
    n_steps = 3
    iters, times, states = run_loop(ehdg, inst, n_steps, loop="persistent")
    assert np.all(times > 0)
    for i, (kw, prob, u0, g) in enumerate(inst):
        args = dict(kw)
        mesh = args.pop("mesh")
        p = args.pop("p")
        with ehdg.Solver(mesh, p, **args) as s:
            s.set_boundary(g)
            s.set_state(u0)
            solo_iters = s.run(n_steps)
            u, uh = s.get_state()
        assert list(iters[i]) == solo_iters, (i, kw["precision"])
        assert np.array_equal(states[i][0], u), (i, kw["precision"])
        assert np.array_equal(states[i][1], uh), (i, kw["precision"])


def test_persistent_loop_with_many_tiles_equals_the_loop(ehdg):
    """Instances of up to 128 tiles each, FP64 and FP32 corrections: the
    persistent form and the loop of launches agree bit for bit over two
    steps (the ring is reused across steps)."""
    rng = np.random.default_rng(42)
    inst = []
    for i in range(20):
        n = int(rng.integers(24, 129))
        p = 1 + i % 5
        th = rng.uniform(0.05, 1.5) + (np.pi / 2) * (i % 4)
        beta = rng.uniform(0.5, 1.5) * np.array([np.cos(th), np.sin(th)])
        mesh = W.structured_mesh((n, n))
        X = node_coords(mesh, p)
        XF = face_point_coords(mesh, p, p + 1)
        kw = dict(mesh=mesh, p=p, scheme="be", dt=0.01, tol=1e-11, max_iter=500,
                  beta_const=beta, precision=("fp64", "fp32")[i % 2], inner_sweeps=3 + i % 4)
        inst.append((kw, None, W.gaussian(X, (0.4, 0.6), 0.1)[:, None, :],
                     W.gaussian(XF, (0.4, 0.6), 0.1)))
    a_iters, _, a_states = run_loop(ehdg, inst, 2, loop="persistent")
    b_iters, _, b_states = run_loop(ehdg, inst, 2, loop=True)
    assert np.array_equal(a_iters, b_iters)
    for (u, uh), (ru, ruh) in zip(a_states, b_states):
        assert np.array_equal(u, ru) and np.array_equal(uh, ruh)


def test_persistent_loop_reports_an_instance_that_does_not_converge(ehdg):
    """An instance that hits max_iter in the persistent form stops with
    EHDG_ERR_NOT_CONVERGED while the others run on to their tolerance."""
    inst = loop_instances(n=5, seed=43, precisions=("fp64", "fp32"))
    kw0 = dict(inst[0][0], tol=1e-30, max_iter=3)
    inst[0] = (kw0,) + inst[0][1:]
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        b.set_loop("persistent")
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        with pytest.raises(ehdg.EhdgError) as ei:
            b.run(1)
        assert ei.value.status == 4
        states = [s.get_state() for s in b.instances]
    for i, (kw, prob, u0, g) in enumerate(inst[1:], start=1):
        ou, _, _, _ = prob.run(u0, 1, g_of_t=lambda t: g, tol=1e-13, max_iter=2000)
        assert np.linalg.norm(states[i][0] - ou) / np.linalg.norm(ou) < 1e-10, i


def test_batched_loop_reports_an_instance_that_does_not_converge(ehdg):
    """An instance that hits max_iter stops with EHDG_ERR_NOT_CONVERGED while
    the others run on to their tolerance."""
    inst = loop_instances(n=4, seed=33, precisions=("fp64", "tf32"))
    kw0 = dict(inst[0][0], tol=1e-30, max_iter=3)
    inst[0] = (kw0,) + inst[0][1:]
    with ehdg.Batch([kw for kw, _, _, _ in inst]) as b:
        for (kw, prob, u0, g), s in zip(inst, b.instances):
            s.set_boundary(g)
            s.set_state(u0)
        with pytest.raises(ehdg.EhdgError) as ei:
            b.run(1)
        assert ei.value.status == 4
        states = [s.get_state() for s in b.instances]
    for i, (kw, prob, u0, g) in enumerate(inst[1:], start=1):
        ou, _, _, _ = prob.run(u0, 1, g_of_t=lambda t: g, tol=1e-13, max_iter=2000)
        assert np.linalg.norm(states[i][0] - ou) / np.linalg.norm(ou) < 1e-10, i
