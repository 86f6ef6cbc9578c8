"""Edge cases of the GPU path against the CPU oracle.

- single elements, whose every face is a boundary face;
- one-element-wide strips, where a 128- or 32-element tile holds a ragged
  handful of elements;
- the highest degrees the library accepts (2D p = 6, 3D p = 3 with a
  variable velocity: 216 face points per element, shallow water p = 5);
- the degenerate velocity beta = 0, where every face point has
  sgn(beta.n) = 0 and the trace formula (eq. transportLocale) is the
  average of the two sides.

FP64 paths match the oracle to 1e-12 relative L2. The mixed-precision
forms reach the FP64 solution to 1e-10 after defect correction.
"""
import zlib

import numpy as np
import pytest

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


def variable_2d(mesh, p):
    wl = W.transport_2d_variable(n=(1, 1), p=p)
    return wl.beta_nodes(node_coords(mesh, p))


def variable_3d(mesh, p):
    X = node_coords(mesh, p)
    b = np.stack([0.6 + 0.2 * X[..., 1], -0.5 + 0.3 * X[..., 2], 0.4 + 0.2 * X[..., 0]], -1)
    return np.ascontiguousarray(np.transpose(b, (0, 2, 1)))


def make_case(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "2d_single_element":
        mesh, p = W.structured_mesh((1, 1)), 2
        kw = dict(scheme="be", dt=0.02, beta_const=np.array([1.0, 0.5]))
    elif name == "2d_single_element_variable":
        mesh, p = W.structured_mesh((1, 1)), 3
        kw = dict(scheme="cn", dt=0.01, beta_nodes=variable_2d(mesh, 3))
    elif name == "2d_strip_variable":
        mesh, p = W.structured_mesh((1, 29)), 2
        kw = dict(scheme="cn", dt=0.01, beta_nodes=variable_2d(mesh, 2))
    elif name == "2d_strip_const":
        mesh, p = W.structured_mesh((37, 1)), 1
        kw = dict(scheme="be", dt=0.02, beta_const=np.array([-0.3, 0.9]))
    elif name == "2d_max_degree_const":
        mesh, p = W.structured_mesh((5, 4)), 6
        kw = dict(scheme="be", dt=0.02, beta_const=np.array([0.7, -0.4]))
    elif name == "2d_max_degree_variable":
        mesh, p = W.structured_mesh((5, 4)), 6
        kw = dict(scheme="cn", dt=0.01, beta_nodes=variable_2d(mesh, 6))
    elif name == "3d_single_element":
        mesh, p = W.structured_mesh((1, 1, 1)), 3
        kw = dict(scheme="be", dt=5e-3, beta_const=np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0))
    elif name == "3d_max_degree_variable":
        mesh, p = W.structured_mesh((3, 2, 2)), 3
        kw = dict(scheme="be", dt=0.05, beta_nodes=variable_3d(mesh, 3))
    elif name == "2d_zero_velocity":
        mesh, p = W.structured_mesh((6, 5)), 2
        kw = dict(scheme="be", dt=0.02, beta_const=np.zeros(2))
    elif name == "3d_zero_velocity":
        mesh, p = W.structured_mesh((3, 3, 2)), 2
        kw = dict(scheme="be", dt=0.05, beta_const=np.zeros(3))
    elif name == "sw_single_element":
        mesh, p = W.structured_mesh((1, 1), boundary_tag=W.TAG_WALL), 2
        kw = dict(pde="sw", scheme="be", dt=2e-3, Phi=1.3)
    elif name == "sw_max_degree":
        mesh, p = W.structured_mesh((4, 3), boundary_tag=W.TAG_WALL), 5
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


CASES = ["2d_single_element", "2d_single_element_variable", "2d_strip_variable",
         "2d_strip_const", "2d_max_degree_const", "2d_max_degree_variable",
         "3d_single_element", "3d_max_degree_variable", "2d_zero_velocity", "3d_zero_velocity",
         "sw_single_element", "sw_max_degree"]
# one local operator for every element: the tensor-core forms apply
SHARED = ["2d_single_element", "2d_strip_const", "2d_max_degree_const", "3d_single_element",
          "2d_zero_velocity", "3d_zero_velocity", "sw_single_element", "sw_max_degree"]


def solver(E, mesh, p, kw, tol=1e-10, max_iter=400, **extra):
    return E.Solver(mesh, p, tol=tol, max_iter=max_iter, **dict(kw, **extra))


def oracle_run(prob, u0, g, n_steps, tol):
    return prob.run(u0, n_steps, g_of_t=(None if g is None else (lambda t: g)), tol=tol)


@pytest.mark.parametrize("name", CASES)
def test_fixed_iterations_match_oracle(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_iter = 3
    with solver(ehdg, mesh, p, kw) as s:
        assert s.info["Nqf"] == prob.Nqf
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        s.step_fixed(n_iter)
        u, uh = s.get_state()
        hist = s.residual_history()
    uhn = prob.trace(u0, g)
    ou, ouh, ohist = prob.solve_step(u0, uhn, g_new=g, fixed_iters=n_iter)
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL
    assert len(hist) == n_iter
    # residuals at the rounding level (beta = 0) agree only in magnitude
    scale = np.sqrt(np.sum(prob.face_w * ouh * ouh))
    assert np.allclose(hist, ohist, rtol=1e-9, atol=1e-13 * scale)


@pytest.mark.parametrize("name", CASES)
def test_steps_to_tolerance_match_oracle(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 2
    with solver(ehdg, mesh, p, kw) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = oracle_run(prob, u0, g, n_steps, 1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL
    if "zero_velocity" in name:
        # beta = 0: the state does not move and one iteration ends each step
        assert iters == [1] * n_steps
        assert rel(u, u0) < 1e-13


@pytest.mark.parametrize("name", SHARED)
def test_fp64_emulated_matches_oracle(ehdg, name):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 2
    with solver(ehdg, mesh, p, kw, precision="fp64_emulated") as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        iters = s.run(n_steps)
        u, uh = s.get_state()
    ou, ouh, oiters, _ = oracle_run(prob, u0, g, n_steps, 1e-10)
    assert iters == oiters
    assert rel(u, ou) < RTOL
    assert rel(uh, ouh) < RTOL


def mixed_forms():
    out = [(n, "fp32") for n in CASES]
    out += [(n, pr) for n in SHARED for pr in ("tf32", "bf16")]
    return out


@pytest.mark.parametrize("name,precision", mixed_forms())
def test_mixed_precision_reaches_fp64_solution(ehdg, name, precision):
    mesh, p, kw, prob, u0, g = make_case(name)
    n_steps = 2
    with solver(ehdg, mesh, p, kw, tol=1e-12, precision=precision, inner_sweeps=4) as s:
        if g is not None:
            s.set_boundary(g)
        s.set_state(u0)
        s.run(n_steps)
        u, uh = s.get_state()
    ou, ouh, _, _ = oracle_run(prob, u0, g, n_steps, 1e-13)
    assert rel(u, ou) < 1e-10, precision
    assert rel(uh, ouh) < 1e-10, precision


def test_zero_steps_leave_the_state(ehdg):
    mesh, p, kw, prob, u0, g = make_case("2d_strip_variable")
    with solver(ehdg, mesh, p, kw) as s:
        s.set_boundary(g)
        s.set_state(u0)
        a = s.get_state()
        assert s.run(0) == []
        b = s.get_state()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_batch_of_one_equals_solo_run(ehdg):
    mesh, p, kw, prob, u0, g = make_case("2d_single_element_variable")
    spec = dict(kw, mesh=mesh, p=p, tol=1e-10, max_iter=400)
    with ehdg.Batch([spec]) as b:
        s = b.instances[0]
        s.set_boundary(g)
        s.set_state(u0)
        iters, times = b.run(3)
        ub, uhb = s.get_state()
    with solver(ehdg, mesh, p, kw) as s:
        s.set_boundary(g)
        s.set_state(u0)
        solo = s.run(3)
        u, uh = s.get_state()
    assert list(iters[0]) == solo and times[0] > 0
    assert np.array_equal(ub, u) and np.array_equal(uhb, uh)
