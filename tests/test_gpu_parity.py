"""GPU path (through the C ABI) against the CPU oracle, element by element.

Sizes span several thread blocks with a ragged tail; tolerances: relative L2
1e-12 in float64 (the float64 target of the method's GPU path).
"""
import zlib

import numpy as np
import pytest

from oracle import direct
from oracle.ehdg import Problem
from oracle.geometry import face_point_coords, node_coords
from paper_1601_06681_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def ehdg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_06681_gb300 import build, ehdg as E
    build.build()
    E.load()
    return E


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def make_case(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "2d_be_const":
        mesh, p = W.structured_mesh((17, 11)), 2
        kw = dict(scheme="be", dt=0.02, beta_const=np.array([1.0, 0.5]))
    elif name == "2d_be_zero_component":
        mesh, p = W.structured_mesh((13, 10)), 3
        kw = dict(scheme="be", dt=0.05, beta_const=np.array([-0.8, 0.0]))
    elif name == "2d_cn_variable":
        wl = W.transport_2d_variable(n=(14, 11), p=3)
        mesh, p = wl.mesh(), 3
        kw = dict(scheme="cn", dt=0.01, beta_nodes=wl.beta_nodes(node_coords(mesh, p)))
    elif name == "2d_cn_variable_p4":
        wl = W.transport_2d_variable(n=(12, 12), p=4)
        mesh, p = wl.mesh(), 4
        kw = dict(scheme="cn", dt=2e-3, beta_nodes=wl.beta_nodes(node_coords(mesh, p)))
    elif name == "2d_steady_variable":
        mesh, p = W.structured_mesh((9, 8)), 2
        X = node_coords(mesh, p)
        bn = np.ascontiguousarray(np.transpose(np.stack([X[..., 1] + 0.1, X[..., 0] + 0.2], -1), (0, 2, 1)))
        kw = dict(scheme="steady", beta_nodes=bn)
    elif name == "2d_graded_mesh":
        # conforming mesh with graded spacing: per-element operators, constant beta
        nx, ny = 10, 13
        mesh, p = W.structured_mesh((nx, ny)), 2
        xs = (np.arange(nx + 1) / nx) ** 1.4
        ys = np.sin(0.5 * np.pi * np.arange(ny + 1) / ny)
        i0 = np.arange(mesh["n_elem"]) % nx
        i1 = np.arange(mesh["n_elem"]) // nx
        mesh["elem_lo"] = np.stack([xs[i0], ys[i1]], -1)
        mesh["elem_h"] = np.stack([xs[i0 + 1] - xs[i0], ys[i1 + 1] - ys[i1]], -1)
        kw = dict(scheme="be", dt=0.03, beta_const=np.array([0.6, -0.9]))
    elif name == "2d_per_element_const_beta":
        # a constant velocity given per node takes the per-element path
        mesh, p = W.structured_mesh((10, 13)), 2
        kw = dict(scheme="be", dt=0.03, beta_nodes=np.ascontiguousarray(
            np.broadcast_to(np.array([0.6, -0.9])[None, :, None], (mesh["n_elem"], 2, (p + 1) ** 2))))
    elif name == "2d_per_element_tangent":
        # per-node constant velocity with beta.n = 0 on every horizontal face:
        # the per-element sweep plus the finishing kernel of tangential points
        mesh, p = W.structured_mesh((11, 9)), 3
        kw = dict(scheme="be", dt=0.04, beta_nodes=np.ascontiguousarray(
            np.broadcast_to(np.array([-0.8, 0.0])[None, :, None], (mesh["n_elem"], 2, (p + 1) ** 2))))
    elif name == "3d_be_variable":
        # hexahedra with per-node velocity (per-element operators, 3x3 points per face)
        mesh, p = W.structured_mesh((5, 4, 3)), 1
        X = node_coords(mesh, p)
        b = np.stack([0.6 + 0.2 * X[..., 1], -0.5 + 0.3 * X[..., 2], 0.4 + 0.2 * X[..., 0]], -1)
        kw = dict(scheme="be", dt=0.05, beta_nodes=np.ascontiguousarray(np.transpose(b, (0, 2, 1))))
    elif name == "3d_be_variable_p2":
        # per-node velocity with 5x5 points per face: the fused per-element sweep
        mesh, p = W.structured_mesh((4, 3, 3)), 2
        X = node_coords(mesh, p)
        b = np.stack([0.6 + 0.2 * X[..., 1], -0.5 + 0.3 * X[..., 2], 0.4 + 0.2 * X[..., 0]], -1)
        kw = dict(scheme="be", dt=0.05, beta_nodes=np.ascontiguousarray(np.transpose(b, (0, 2, 1))))
    elif name == "3d_be_const":
        mesh, p = W.structured_mesh((6, 5, 4)), 2
        kw = dict(scheme="be", dt=0.05, beta_const=np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0))
    elif name == "3d_be_const_p3":
        mesh, p = W.structured_mesh((5, 3, 4)), 3
        kw = dict(scheme="be", dt=5e-3, beta_const=np.array([0.3, -1.0, 0.6]))
    elif name == "3d_be_const_p3_tiles":
        # 360 elements: two full 128-element tiles and a ragged third
        mesh, p = W.structured_mesh((9, 8, 5)), 3
        kw = dict(scheme="be", dt=5e-3, beta_const=np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0))
    elif name == "3d_cn_const_p3":
        # Crank-Nicolson with one shared hexahedral operator (the sum-factorised
        # sweep and its reconstruction 2 v - u^n)
        mesh, p = W.structured_mesh((5, 4, 3)), 3
        kw = dict(scheme="cn", dt=5e-3, beta_const=np.array([0.3, -1.0, 0.6]))
    elif name == "3d_be_const_p1":
        mesh, p = W.structured_mesh((7, 6, 5)), 1
        kw = dict(scheme="be", dt=0.02, beta_const=np.array([-0.5, 0.8, 0.35]))
    elif name == "2d_cn_const":
        # Crank-Nicolson with one shared operator
        mesh, p = W.structured_mesh((15, 12)), 3
        kw = dict(scheme="cn", dt=0.01, beta_const=np.array([0.7, -0.4]))
    elif name == "3d_be_tangent_p2":
        # beta.n = 0 on the y and z faces: tangential rows beside the upwind ones
        mesh, p = W.structured_mesh((7, 5, 4)), 2
        kw = dict(scheme="be", dt=0.02, beta_const=np.array([0.7, 0.0, 0.0]))
    elif name == "sw_be":
        mesh, p = W.structured_mesh((12, 11), boundary_tag=W.TAG_WALL), 2
        kw = dict(pde="sw", scheme="be", dt=2e-3, Phi=1.3)
    elif name == "sw_fplane":
        # Coriolis f-plane and bottom friction: still one shared operator
        mesh, p = W.structured_mesh((12, 11), boundary_tag=W.TAG_WALL), 2
        kw = dict(pde="sw", scheme="be", dt=2e-3, Phi=1.3, coriolis=(0.9, 0.0, 0.0),
                  friction=0.2)
    elif name == "sw_betaplane":
        # beta-plane Coriolis f = f0 + beta (y - y_m) and friction: per-element operators
        mesh, p = W.structured_mesh((9, 10), boundary_tag=W.TAG_WALL), 3
        kw = dict(pde="sw", scheme="be", dt=1e-3, Phi=1.0, coriolis=(0.5, 2.0, 0.4),
                  friction=0.3)
    elif name == "sw_be_p3":
        mesh, p = W.structured_mesh((9, 14), boundary_tag=W.TAG_WALL), 3
        kw = dict(pde="sw", scheme="be", dt=1e-3, Phi=1.0)
    else:
        raise KeyError(name)
    prob = Problem(mesh, p, **kw)
    u0 = rng.standard_normal((prob.nel, prob.nf, prob.Np))
    g = None
    if prob.pde == "transport":
        XF = face_point_coords(mesh, p, prob.ref.q)
        g = np.cos(2.0 * XF[..., 0] + 0.3) * np.sin(3.0 * XF[..., 1] + 0.1)
        if mesh["dim"] == 3:
            g = g * np.cos(XF[..., 2])
    return mesh, p, kw, prob, u0, g


def make_solver(E, mesh, p, kw, prob, tol=1e-10, max_iter=400):
    args = dict(kw)
    return E.Solver(mesh, p, tol=tol, max_iter=max_iter, **args)


CASES = ["2d_be_const", "2d_be_zero_component", "2d_cn_variable", "2d_cn_variable_p4",
         "2d_steady_variable", "2d_graded_mesh", "2d_per_element_const_beta",
         "2d_per_element_tangent", "3d_be_const", "3d_be_const_p3", "3d_be_variable", "sw_be",
         "sw_be_p3", "sw_fplane", "sw_betaplane", "3d_cn_const_p3", "3d_be_const_p1"]


@pytest.mark.parametrize("name", CASES)
def test_coordinates_match_oracle(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        assert np.abs(s.node_coords() - node_coords(mesh, p)).max() < 1e-15
        assert np.abs(s.face_point_coords() - face_point_coords(mesh, p, prob.ref.q)).max() < 1e-15
        assert s.info["Nqf"] == prob.Nqf


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("n_iter", [1, 4])
def test_fixed_iterations_match_oracle(ehdg, name, n_iter):
    mesh, p, kw, prob, u0, g = make_case(name)
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        _, uh0 = s.get_state()
        uhn = prob.trace(u0, g)
        assert rel(uh0, uhn) < RTOL
        s.step_fixed(n_iter)
        u, uh = s.get_state()
        hist = s.residual_history()
    ou, ouh, ohist = prob.solve_step(u0, uhn, g_new=g, fixed_iters=n_iter)
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL
    assert len(hist) == n_iter
    assert np.allclose(hist, ohist, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("name", ["2d_be_const", "2d_cn_variable", "3d_be_const", "sw_be",
                                  "sw_fplane", "sw_betaplane", "3d_cn_const_p3", "3d_be_const_p1"])
def test_steps_to_tolerance_match_oracle(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 3
    with make_solver(ehdg, mesh, p, kw, prob, tol=1e-10) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL


@pytest.mark.parametrize("name, precision", [("3d_be_const_p3", "fp64"),
                                             ("3d_be_const_p3", "fp64_emulated"),
                                             ("3d_be_const_p3", "bf16"),
                                             ("3d_be_variable", "fp64"),
                                             ("3d_be_const_p1", "fp64"),
                                             ("sw_be", "fp64"),
                                             ("sw_be_p3", "fp64_emulated"),
                                             ("sw_fplane", "bf16"),
                                             ("sw_betaplane", "fp64")])
def test_warm_start_of_the_initial_trace_equals_a_cold_start(ehdg, name, precision):
    """3D backward Euler (and shallow water): from the second step on, the
    initial trace is the previous step's final trace (the last sweep wrote
    Ey u^n at every owned point) with the inflow boundary points recomputed. Starting every step
    cold (set_state, which forms the trace formula of u^n) gives the same
    iteration counts and the same state up to rounding."""
    mesh, p, kw, prob, u0, g = make_case(name)
    kw = dict(kw, precision=precision)
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        assert s.info["warm_start"] == 1
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        it_warm = s.run(3)
        uw, uhw = s.get_state()
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        it_cold = []
        for _ in range(3):
            it_cold += s.run(1)
            u, _ = s.get_state()
            s.set_state(u)
        uc, uhc = s.get_state()
    assert it_warm == it_cold
    assert rel(uw, uc) < 1e-13 and rel(uhw, uhc) < 1e-13


def test_warm_start_is_off_where_the_trace_formula_needs_both_sides(ehdg):
    """Crank-Nicolson, points with beta.n = 0, and 2D keep the cold start."""
    for name in ("3d_cn_const_p3", "3d_be_tangent_p2", "2d_be_const"):
        mesh, p, kw, prob, u0, g = make_case(name)
        with make_solver(ehdg, mesh, p, kw, prob) as s:
            assert s.info["warm_start"] == 0, name


def test_autotuner_restores_the_warm_start(ehdg):
    """The inner-sweep autotuner restores the warm-start flag with the rest of
    the state, from a cold state (just after set_state) and from a warm one
    (after a step): runs with autotuner calls in between equal a plain run bit
    for bit (a flag left wrong would change the initial trace's rounding)."""
    mesh, p, kw, prob, u0, g = make_case("3d_be_const_p3")
    kw = dict(kw, precision="bf16", inner_sweeps=4)
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        s.set_boundary(g)
        s.set_state(u0)
        ref_iters = s.run(3)
        ref = s.get_state()
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        s.set_boundary(g)
        s.set_state(u0)
        assert s.autotune_inner_sweeps((4,))[0] == 4      # from a cold state
        iters = s.run(1)
        assert s.autotune_inner_sweeps((4,))[0] == 4      # from a warm state
        iters += s.run(2)
        got = s.get_state()
    assert iters == ref_iters
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_converged_step_equals_direct_hdg_solve(ehdg):
    mesh, p, kw, prob, u0, g = make_case("2d_be_const")
    with make_solver(ehdg, mesh, p, kw, prob, tol=1e-13, max_iter=2000) as s:
        s.set_boundary(g)
        s.set_state(u0)
        s.step()
        u, uh = s.get_state()
    ud, uhd = direct.solve(prob, u0, None, g=g)
    assert rel(u, ud) < 1e-11
    assert rel(uh, uhd) < 1e-11


# "2d_cn_variable" (per-element operator, no beta.n = 0 point) runs every
# iteration of a step in one persistent launch; "2d_be_const" launches one
# sweep per iteration
@pytest.mark.parametrize("name", ["2d_be_const", "2d_cn_variable"])
def test_not_converged_status_keeps_state(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    with make_solver(ehdg, mesh, p, kw, prob, tol=1e-30, max_iter=3) as s:
        s.set_boundary(g)
        s.set_state(u0)
        it, res, st = s.step(check=False)
        assert st == 4 and it == 3
        u, _ = s.get_state()
        hist = s.residual_history()
    ou, _, ohist = prob.solve_step(u0, prob.trace(u0, g), g_new=g, fixed_iters=3)
    assert rel(u, ou) < RTOL
    assert np.allclose(hist[:3], ohist, rtol=1e-9, atol=0)


def test_persistent_step_equals_per_iteration_sweeps(ehdg):
    """A converged step (one launch for all iterations) and the same number
    of iterations launched one by one give the same state, bit for bit."""
    mesh, p, kw, prob, u0, g = make_case("2d_cn_variable")
    with make_solver(ehdg, mesh, p, kw, prob, tol=1e-11, max_iter=400) as s:
        s.set_boundary(g)
        s.set_state(u0)
        it, _, _ = s.step()
        ua, uha = s.get_state()
        s.set_boundary(g)
        s.set_state(u0)
        s.step_fixed(it)
        ub, uhb = s.get_state()
    assert it > 3
    assert np.array_equal(ua, ub)
    assert np.array_equal(uha, uhb)


@pytest.mark.parametrize("name", ["2d_be_const", "2d_cn_variable"])
def test_nan_input_reports_divergence(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    bad = u0.copy()
    bad[3, 0, 1] = np.nan
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        s.set_boundary(g)
        s.set_state(bad)
        it, res, st = s.step(check=False)
        assert st == 5 and it == 1


def test_invalid_arguments_rejected(ehdg):
    mesh = W.structured_mesh((4, 4))
    with pytest.raises(ehdg.EhdgError) as ei:
        ehdg.Solver(mesh, 2, beta_const=[1.0, 0.0], dt=-1.0)
    assert ei.value.status == 1
    bad = dict(mesh)
    bad["face_elem"] = mesh["face_elem"].copy()
    bad["face_elem"][5, 0] = 10 ** 6
    with pytest.raises(ehdg.EhdgError):
        ehdg.Solver(bad, 2, beta_const=[1.0, 0.0], dt=0.1)
    with pytest.raises(ehdg.EhdgError) as ei:
        ehdg.Solver(mesh, 9, beta_const=[1.0, 0.0], dt=0.1)
    assert ei.value.status == 7


def test_device_pointer_io_matches_host_io(ehdg):
    import torch
    mesh, p, kw, prob, u0, g = make_case("2d_cn_variable")
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        s.set_boundary(torch.from_numpy(g).cuda())
        s.set_state(torch.from_numpy(u0).cuda())
        s.step()
        du = torch.empty(s.state_shape, dtype=torch.float64, device="cuda")
        duh = torch.empty(s.trace_shape, dtype=torch.float64, device="cuda")
        s.get_state(du, duh)
        u, uh = s.get_state()
    assert np.array_equal(du.cpu().numpy(), u)
    assert np.array_equal(duh.cpu().numpy(), uh)


# ---------------------------------------------------------------------------
# mixed precision: FP32 inner sweeps + FP64 defect correction
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["2d_be_const", "2d_be_zero_component", "2d_cn_variable",
                                  "2d_cn_variable_p4", "3d_be_const", "sw_be", "2d_graded_mesh",
                                  "2d_per_element_tangent", "3d_be_variable", "sw_betaplane"])
def test_mixed_precision_reaches_fp64_solution(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 3
    args = dict(kw)
    with ehdg.Solver(mesh, p, tol=1e-12, max_iter=400, precision="fp32", inner_sweeps=6,
                     **args) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
        hist = s.residual_history()
    ou, ouh, oiters, _ = prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-13, max_iter=2000)
    assert hist[-1] < 1e-12
    assert rel(u, ou) < 1e-10
    assert rel(uh, ouh) < 1e-10
    # the correction makes every FP64 sweep count for several
    assert sum(iters) < sum(oiters)


def test_mixed_fixed_iterations_are_deterministic(ehdg):
    mesh, p, kw, prob, u0, g = make_case("2d_cn_variable")
    outs = []
    for _ in range(2):
        with ehdg.Solver(mesh, p, tol=1e-10, max_iter=50, precision="fp32", **kw) as s:
            s.set_boundary(g)
            s.set_state(u0)
            s.step_fixed(3)
            outs.append(s.get_state())
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


# ---------------------------------------------------------------------------
# tensor-core (tcgen05) correction sweeps: TF32 and BF16 operands, FP32 accumulate
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["tf32", "bf16"])
@pytest.mark.parametrize("name", ["2d_be_const", "2d_be_zero_component", "3d_be_const",
                                  "3d_be_const_p3", "sw_be_p3", "sw_fplane"])
def test_tensor_core_mixed_reaches_fp64_solution(ehdg, name, precision):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 2
    with ehdg.Solver(mesh, p, tol=1e-12, max_iter=400, precision=precision, inner_sweeps=6,
                     **kw) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-13, max_iter=2000)
    assert rel(u, ou) < 1e-10
    assert rel(uh, ouh) < 1e-10
    assert sum(iters) < sum(oiters)


def test_tf32_precision_needs_shared_operator(ehdg):
    mesh, p, kw, prob, u0, g = make_case("2d_cn_variable")
    with pytest.raises(ehdg.EhdgError) as ei:
        ehdg.Solver(mesh, p, precision="tf32", **kw)
    assert ei.value.status == 7


# per-element operators: BF16 copy of the tile-major operator, FP32 arithmetic
@pytest.mark.parametrize("name", ["2d_cn_variable", "2d_cn_variable_p4", "3d_be_variable",
                                  "2d_per_element_tangent"])
def test_bf16_per_element_mixed_reaches_fp64_solution(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 3
    with ehdg.Solver(mesh, p, tol=1e-12, max_iter=400, precision="bf16", inner_sweeps=6,
                     **dict(kw)) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
        hist = s.residual_history()
    ou, ouh, oiters, _ = prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-13, max_iter=2000)
    assert hist[-1] < 1e-12
    assert rel(u, ou) < 1e-10
    assert rel(uh, ouh) < 1e-10
    assert sum(iters) < sum(oiters)


# ---------------------------------------------------------------------------
# checkpoint / resume and the autotuner
# ---------------------------------------------------------------------------

# "3d_be_const_p3" starts its steps warm (the checkpoint carries that flag)
@pytest.mark.parametrize("name", ["2d_cn_variable", "sw_be", "3d_be_const_p3"])
def test_checkpoint_resume_is_bitwise(ehdg, name, tmp_path):
    mesh, p, kw, prob, u0, g = make_case(name)
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        s.run(4)
        u_ref, uh_ref = s.get_state()
    path = str(tmp_path / "ck.ehdg")
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        s.run(2)
        s.save(path)
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        s.load_checkpoint(path)
        s.run(2)
        u, uh = s.get_state()
    assert np.array_equal(u, u_ref) and np.array_equal(uh, uh_ref)
    # a checkpoint of another problem is rejected
    other = W.structured_mesh((5, 5), boundary_tag=mesh["face_tag"].max())
    kw2 = dict(kw)
    if "beta_nodes" in kw2:
        kw2.pop("beta_nodes")
        kw2["beta_const"] = np.array([1.0, 0.0])
    with ehdg.Solver(other, p, **kw2) as s:
        with pytest.raises(ehdg.EhdgError):
            s.load_checkpoint(path)
    # same mesh, degree and time step, another velocity field: rejected too
    if "beta_nodes" in kw:
        kw3 = dict(kw)
        kw3["beta_nodes"] = np.ascontiguousarray(kw["beta_nodes"] * 1.01)
        with ehdg.Solver(mesh, p, **kw3) as s:
            with pytest.raises(ehdg.EhdgError):
                s.load_checkpoint(path)


def test_autotuner_keeps_state_and_results(ehdg, tmp_path):
    mesh, p, kw, prob, u0, g = make_case("3d_be_const")
    with ehdg.Solver(mesh, p, tol=1e-12, max_iter=400, precision="tf32", **kw) as s:
        s.set_boundary(g)
        s.set_state(u0)
        best = ehdg.autotune_cached(s, str(tmp_path / "tune.json"), candidates=(2, 4, 8))
        assert best in (2, 4, 8)
        s.run(2)
        u, _ = s.get_state()
        again = ehdg.autotune_cached(s, str(tmp_path / "tune.json"))
        assert again == best
    ou, _, _, _ = prob.run(u0, 2, g_of_t=lambda t: g, tol=1e-13, max_iter=2000)
    assert rel(u, ou) < 1e-10


# ---------------------------------------------------------------------------
# FP64-accurate sweeps on the BF16 tensor cores (Ozaki splitting): same
# tolerances as the FP64 path
# ---------------------------------------------------------------------------

OZAKI_CASES = ["2d_be_const", "2d_be_zero_component", "2d_cn_const", "3d_be_const",
               "3d_be_const_p3", "3d_be_const_p3_tiles", "3d_be_tangent_p2", "sw_be", "sw_be_p3",
               "sw_fplane"]


@pytest.mark.parametrize("name", OZAKI_CASES)
@pytest.mark.parametrize("n_iter", [1, 4])
def test_fp64_emulated_fixed_iterations_match_oracle(ehdg, name, n_iter):
    mesh, p, kw, prob, u0, g = make_case(name)
    with ehdg.Solver(mesh, p, tol=1e-10, max_iter=400, precision="fp64_emulated", **kw) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        s.step_fixed(n_iter)
        u, uh = s.get_state()
        hist = s.residual_history()
    ou, ouh, ohist = prob.solve_step(u0, prob.trace(u0, g), g_new=g, fixed_iters=n_iter)
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL
    assert len(hist) == n_iter
    assert np.allclose(hist, ohist, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("name", OZAKI_CASES)
def test_fp64_emulated_steps_to_tolerance_match_oracle(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 3
    with ehdg.Solver(mesh, p, tol=1e-10, max_iter=400, precision="fp64_emulated", **kw) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL


def test_fp64_emulated_converged_step_equals_direct_hdg_solve(ehdg):
    mesh, p, kw, prob, u0, g = make_case("3d_be_const")
    with ehdg.Solver(mesh, p, tol=1e-13, max_iter=2000, precision="fp64_emulated", **kw) as s:
        s.set_boundary(g)
        s.set_state(u0)
        s.step()
        u, uh = s.get_state()
    ud, uhd = direct.solve(prob, u0, None, g=g)
    assert rel(u, ud) < 1e-11
    assert rel(uh, uhd) < 1e-11


def test_fp64_emulated_nan_input_reports_divergence(ehdg):
    mesh, p, kw, prob, u0, g = make_case("3d_be_const")
    bad = u0.copy()
    bad[7, 0, 2] = np.nan
    with ehdg.Solver(mesh, p, tol=1e-10, max_iter=400, precision="fp64_emulated", **kw) as s:
        s.set_boundary(g)
        s.set_state(bad)
        it, res, st = s.step(check=False)
        assert st == 5 and it == 1


def test_fp64_emulated_rejects_unsupported_problems(ehdg):
    # per-element operators (variable velocity; beta-plane), and more than 64 sweep rows
    for name in ("2d_cn_variable", "sw_betaplane"):
        mesh, p, kw, prob, u0, g = make_case(name)
        with pytest.raises(ehdg.EhdgError) as ei:
            ehdg.Solver(mesh, p, precision="fp64_emulated", **kw)
        assert ei.value.status == 7
    mesh = W.structured_mesh((3, 3, 3))
    with pytest.raises(ehdg.EhdgError) as ei:
        ehdg.Solver(mesh, 3, scheme="be", dt=0.01, beta_const=[1.0, 0.0, 0.0],
                    precision="fp64_emulated")
    assert ei.value.status == 7


# mixed precision whose outer FP64 sweeps run on the tensor cores (Ozaki)
@pytest.mark.parametrize("precision", ["bf16", "tf32", "fp32"])
@pytest.mark.parametrize("name", ["2d_be_const", "3d_be_const", "3d_be_const_p3_tiles",
                                  "3d_be_tangent_p2", "sw_be_p3"])
def test_mixed_with_emulated_outer_sweeps_reaches_fp64_solution(ehdg, name, precision):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 2
    with ehdg.Solver(mesh, p, tol=1e-12, max_iter=400, precision=precision, inner_sweeps=6,
                     emulated_outer=True, **kw) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
        hist = s.residual_history()
    ou, ouh, oiters, _ = prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-13, max_iter=2000)
    assert hist[-1] < 1e-12
    assert rel(u, ou) < 1e-10
    assert rel(uh, ouh) < 1e-10
    assert sum(iters) < sum(oiters)


def test_emulated_outer_sweeps_need_a_shared_operator(ehdg):
    mesh, p, kw, prob, u0, g = make_case("2d_cn_variable")
    with pytest.raises(ehdg.EhdgError) as ei:
        ehdg.Solver(mesh, p, precision="bf16", emulated_outer=True, **kw)
    assert ei.value.status == 7


# a forcing term f in the step's right-hand side (Crank-Nicolson averages the
# two levels), on the DFMA and on the tensor-core step
@pytest.mark.parametrize("precision", ["fp64", "fp64_emulated"])
@pytest.mark.parametrize("name", ["2d_cn_const", "3d_be_const"])
def test_forcing_matches_oracle(ehdg, name, precision):
    mesh, p, kw, prob, u0, g = make_case(name)
    f = np.random.default_rng(zlib.crc32(b"forcing" + name.encode())).standard_normal(
        (prob.nel, prob.nf, prob.Np))
    with ehdg.Solver(mesh, p, tol=1e-10, max_iter=400, precision=precision, **kw) as s:
        s.set_boundary(g)
        s.set_state(u0)
        s.set_forcing(f)
        iters = s.run(3)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = prob.run(u0, 3, g_of_t=lambda t: g, f_of_t=lambda t: f, tol=1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL


# the FP64-path autotuner: both paths are FP64-accurate, the state is untouched
@pytest.mark.parametrize("name", ["3d_be_const_p3_tiles", "2d_be_const", "sw_be"])
def test_fp64_path_autotuner_keeps_state_and_results(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    with ehdg.Solver(mesh, p, tol=1e-10, max_iter=400, precision="fp64_emulated", **kw) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        before = s.get_state()
        tc, ms_dfma, ms_tensor = s.autotune_fp64_path()
        assert ms_dfma > 0 and ms_tensor > 0 and tc == (ms_tensor < ms_dfma)
        after = s.get_state()
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        iters = s.run(2)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = prob.run(u0, 2, g_of_t=(None if g is None else (lambda t: g)),
                                  tol=1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL
    with ehdg.Solver(mesh, p, precision="fp64", **kw) as s:
        with pytest.raises(ehdg.EhdgError) as ei:
            s.autotune_fp64_path()
        assert ei.value.status == 1


# the tile-shape autotuner of the fused and the sum-factorised FP64 sweeps: FT
# row groups per 32-element tile change which thread runs which row, not the
# rows' arithmetic
@pytest.mark.parametrize("name", ["3d_be_const", "3d_be_variable_p2", "2d_be_zero_component"])
def test_sweep_tile_choice_keeps_iterates_bitwise(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    states = []
    with make_solver(ehdg, mesh, p, kw, prob) as s:
        for ft in (2, 4, 8):
            s.set_boundary(g)
            s.set_state(u0)
            before = s.get_state()
            best, ms = s.autotune_sweep_tile((ft,))
            assert best == ft and ms > 0
            after = s.get_state()
            assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
            s.step_fixed(5)
            states.append(s.get_state())
        best, _ = s.autotune_sweep_tile()
        assert best in (2, 4, 8)
        s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(2)
        u, uh = s.get_state()
    for a, b in zip(states[1:], states[:-1]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ou, ouh, oiters, _ = prob.run(u0, 2, g_of_t=lambda t: g, tol=1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL


def test_sweep_tile_autotuner_rejects_other_sweeps(ehdg):
    # shallow water; the tiled per-element sweeps of quadrilaterals and of 2x2-point
    # hexahedra; the one-thread-per-element sweep of quadrilaterals with a shared operator
    for name in ("sw_be", "2d_cn_variable", "3d_be_variable", "2d_be_const"):
        mesh, p, kw, prob, u0, g = make_case(name)
        with make_solver(ehdg, mesh, p, kw, prob) as s:
            with pytest.raises(ehdg.EhdgError) as ei:
                s.autotune_sweep_tile()
            assert ei.value.status == 1
