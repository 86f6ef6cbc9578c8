"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The benchmark workload (2D transport, 256 x 256 quads, p = 4, per-element
velocity, Crank-Nicolson) is too large for the oracle as a whole. After k eHDG
iterations, though, an element's state depends only on elements at most k + 1
rings away. So each sampled output is computed by the oracle on a patch of
(2k + 3) x (2k + 3) elements around the sampled element, clipped to the domain,
and compared with the GPU's full-size run:

- Where the patch meets the domain boundary, it has the true inflow data.
- Its artificial edges get arbitrary data, whose influence stays more than one
  ring away from the centre.
"""
import numpy as np
import pytest

from oracle.ehdg import Problem
from oracle.geometry import face_point_coords, node_coords
from paper_1601_06681_gb300 import workloads as W

N = 256
P = 4
SAMPLES = [(0, 0), (N - 1, 0), (0, N - 1), (N - 1, N - 1), (128, 128), (3, 200), (200, 3),
           (77, N - 1), (N - 2, 141), (31, 32), (95, 160)]


@pytest.fixture(scope="module")
def ehdg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_06681_gb300 import build, ehdg as E
    build.build()
    E.load()
    return E


@pytest.mark.parametrize("k", [1, 2])
def test_patch_oracle_equals_whole_mesh_oracle(k):
    """The patch argument itself, on a mesh small enough for the whole-mesh
    oracle: every element's patch result equals the whole-mesh result."""
    n = 9
    wl = W.transport_2d_variable(n=(n, n), p=P)
    mesh = W.structured_mesh((n, n))
    X = node_coords(mesh, P)
    prob = Problem(mesh, P, scheme="cn", dt=wl.dt, beta_nodes=wl.beta_nodes(X))
    u0 = wl.initial(X)
    g = wl.boundary(face_point_coords(mesh, P, prob.ref.q), 0.0)
    u, uh, _ = prob.solve_step(u0, prob.trace(u0, g), g, fixed_iters=k)
    for cj in range(n):
        for ci in range(n):
            e = cj * n + ci
            up, uhp = patch_solve(wl, mesh, u0, ci, cj, k, N=n)
            assert np.linalg.norm(up - u[e]) <= 1e-13 * max(np.linalg.norm(u[e]), 1e-3)
            assert np.linalg.norm(uhp - uh[mesh["elem_face"][e]]) <= 1e-13 * max(
                np.linalg.norm(uh[mesh["elem_face"][e]]), 1e-3)


@pytest.fixture(scope="module")
def full_run(ehdg):
    """GPU outputs of one Crank-Nicolson step with 1 and with 2 iterations."""
    wl = W.transport_2d_variable(n=(N, N), p=P)
    mesh = W.structured_mesh((N, N))
    X = node_coords(mesh, P)
    beta = wl.beta_nodes(X)
    u0 = wl.initial(X)
    out = {}
    with ehdg.Solver(mesh, P, scheme="cn", dt=wl.dt, tol=wl.tol, max_iter=100,
                     beta_nodes=beta) as s:
        XF = s.face_point_coords()
        g = wl.boundary(XF, 0.0)
        for k in (1, 2):
            s.set_boundary(g)
            s.set_state(u0)
            s.step_fixed(k)
            out[k] = s.get_state()
    return wl, mesh, u0, out


def patch_solve(wl, mesh, u0, ci, cj, k, N=N):
    """Oracle state and traces of element (ci, cj) of an N x N mesh after k
    iterations of one CN step, from a patch of radius k + 1 around it."""
    r = k + 1
    i0, i1 = max(ci - r, 0), min(ci + r, N - 1)
    j0, j1 = max(cj - r, 0), min(cj + r, N - 1)
    nx, ny = i1 - i0 + 1, j1 - j0 + 1
    h = 1.0 / N
    pm = W.structured_mesh((nx, ny), lo=(i0 * h, j0 * h), hi=((i1 + 1) * h, (j1 + 1) * h))
    Xp = node_coords(pm, P)
    prob = Problem(pm, P, scheme="cn", dt=wl.dt, beta_nodes=wl.beta_nodes(Xp))
    # the patch's elements take the full mesh's initial values
    ii, jj = np.meshgrid(np.arange(i0, i1 + 1), np.arange(j0, j1 + 1), indexing="xy")
    full_ids = (jj * N + ii).reshape(-1)
    up = u0.reshape(N * N, 1, -1)[full_ids]
    # boundary data: the true inflow data on the domain's edges, zero elsewhere
    XFp = face_point_coords(pm, P, prob.ref.q)
    gp = np.zeros((pm["n_face"], prob.Nqf))
    true_g = wl.boundary(XFp, 0.0)
    for f in range(pm["n_face"]):
        if pm["face_elem"][f, 1] >= 0:
            continue
        c = XFp[f].mean(axis=0)
        on_edge = min(c[0], 1.0 - c[0], c[1], 1.0 - c[1]) < 0.25 * h
        if on_edge:
            gp[f] = true_g[f]
    u, uh, _ = prob.solve_step(up, prob.trace(up, gp), gp, fixed_iters=k)
    ep = (cj - j0) * nx + (ci - i0)
    return u[ep], uh[pm["elem_face"][ep]]


@pytest.mark.gpu
@pytest.mark.parametrize("k", [1, 2])
def test_full_size_sampled_elements_match_oracle(full_run, k):
    wl, mesh, u0, out = full_run
    u_gpu, uh_gpu = out[k]
    worst = 0.0
    for ci, cj in SAMPLES:
        u_or, uh_or = patch_solve(wl, mesh, u0, ci, cj, k)
        e = cj * N + ci
        ug = u_gpu.reshape(N * N, 1, -1)[e]
        uhg = uh_gpu[mesh["elem_face"][e]]
        scale = max(np.linalg.norm(u_or), 1e-3)
        err_u = np.linalg.norm(ug - u_or) / scale
        err_t = np.linalg.norm(uhg - uh_or) / max(np.linalg.norm(uh_or), 1e-3)
        worst = max(worst, err_u, err_t)
        assert err_u < 1e-12, (ci, cj, err_u)
        assert err_t < 1e-12, (ci, cj, err_t)
    assert worst < 1e-12


# ---------------------------------------------------------------------------
# 3D transport at its benchmark size: 64^3 hexahedra, p = 3, one operator
# shared by all elements, backward Euler. The native FP64 sweep and the
# FP64-accurate tensor-core sweep (Ozaki splitting) against the oracle on
# patches of (2k + 3)^3 elements.
# ---------------------------------------------------------------------------

N3 = 64
P3 = 3
SAMPLES3 = [(0, 0, 0), (N3 - 1, N3 - 1, N3 - 1), (0, N3 - 1, 31), (31, 32, 33), (N3 - 1, 0, 10),
            (5, 60, N3 - 1), (40, 2, 17)]


@pytest.fixture(scope="module")
def full_run_3d(ehdg):
    wl = W.transport_3d(n=(N3, N3, N3), p=P3)
    mesh = W.structured_mesh((N3, N3, N3))
    u0 = wl.initial(node_coords(mesh, P3))
    out = {}
    for prec in ("fp64", "fp64_emulated"):
        with ehdg.Solver(mesh, P3, scheme="be", dt=wl.dt, tol=wl.tol, max_iter=100,
                         beta_const=wl.beta_const, precision=prec) as s:
            g = wl.boundary(s.face_point_coords(), wl.dt)
            for k in (1, 2):
                s.set_boundary(g)
                s.set_state(u0)
                s.step_fixed(k)
                out[prec, k] = s.get_state()
    return wl, mesh, u0, out


def patch_solve_3d(wl, mesh, u0, c, k):
    """Oracle state and traces of element c = (ci, cj, ck) of the N3^3 mesh
    after k iterations of one backward-Euler step, from a patch of radius
    k + 1 around it (true inflow data on the domain's faces, zero elsewhere)."""
    r = k + 1
    lo = [max(v - r, 0) for v in c]
    hi = [min(v + r, N3 - 1) for v in c]
    n = [hi[a] - lo[a] + 1 for a in range(3)]
    h = 1.0 / N3
    pm = W.structured_mesh(tuple(n), lo=tuple(v * h for v in lo),
                           hi=tuple((v + 1) * h for v in hi))
    prob = Problem(pm, P3, scheme="be", dt=wl.dt, beta_const=wl.beta_const)
    ii, jj, kk = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[2], hi[2] + 1), indexing="ij")
    # patch element ids run x fastest, like the full mesh's
    full_ids = ((kk * N3 + jj) * N3 + ii).transpose(2, 1, 0).reshape(-1)
    up = u0.reshape(N3 ** 3, 1, -1)[full_ids]
    XFp = face_point_coords(pm, P3, prob.ref.q)
    gp = np.zeros((pm["n_face"], prob.Nqf))
    true_g = wl.boundary(XFp, wl.dt)
    for f in range(pm["n_face"]):
        if pm["face_elem"][f, 1] >= 0:
            continue
        x = XFp[f].mean(axis=0)
        if min(x.min(), (1.0 - x).min()) < 0.25 * h:
            gp[f] = true_g[f]
    u, uh, _ = prob.solve_step(up, prob.trace(up, gp), gp, fixed_iters=k)
    ep = ((c[2] - lo[2]) * n[1] + (c[1] - lo[1])) * n[0] + (c[0] - lo[0])
    return u[ep], uh[pm["elem_face"][ep]]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp64_emulated"])
@pytest.mark.parametrize("k", [1, 2])
def test_full_size_3d_sampled_elements_match_oracle(full_run_3d, prec, k):
    wl, mesh, u0, out = full_run_3d
    u_gpu, uh_gpu = out[prec, k]
    for c in SAMPLES3:
        u_or, uh_or = patch_solve_3d(wl, mesh, u0, c, k)
        e = (c[2] * N3 + c[1]) * N3 + c[0]
        ug = u_gpu.reshape(N3 ** 3, 1, -1)[e]
        uhg = uh_gpu[mesh["elem_face"][e]]
        err_u = np.linalg.norm(ug - u_or) / max(np.linalg.norm(u_or), 1e-3)
        err_t = np.linalg.norm(uhg - uh_or) / max(np.linalg.norm(uh_or), 1e-3)
        assert err_u < 1e-12, (c, err_u)
        assert err_t < 1e-12, (c, err_t)
