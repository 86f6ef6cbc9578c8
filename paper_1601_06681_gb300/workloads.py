"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no eHDG arithmetic: it builds structured-mesh connectivity
(an input of the method, Sec. 2: the partition into elements K_j and the
skeleton of unique faces) and draws the random parameters of the analytic
fields used as initial data, velocity fields and boundary data. Field values
are produced by evaluating those analytic functions at physical coordinates
that the caller supplies (each side computes its own node coordinates).

Mesh conventions (shared by every consumer):
  * elements are axis-aligned boxes, numbered e = i0 + N0*(i1 + N1*i2);
  * local faces are f = 2*axis + side (side 0 = low, 1 = high), i.e. the order
    -x, +x, -y, +y, -z, +z;
  * faces are numbered axis by axis; within an axis the face grid
    (N_axis + 1 planes by N_other elements) is flattened with axis 0 fastest;
  * face_elem[e] = (minus, plus): for an interior face, minus is the element on
    the low side, so n^- = +e_axis; for a boundary face, minus is the only
    element and plus = -1; face_local holds the local face index on each side
    (-1 for a missing plus side);
  * face_tag: 0 interior, 1 boundary with Dirichlet data (transport), 2 wall
    (shallow water).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TAG_INTERIOR = 0
TAG_DIRICHLET = 1
TAG_WALL = 2


def structured_mesh(n, lo=None, hi=None, boundary_tag=TAG_DIRICHLET):
    """Connectivity and geometry of an axis-aligned N0 x N1 (x N2) box mesh.

    Returns a dict of numpy arrays: dim, n_elem, n_face, elem_lo [n_elem, dim],
    elem_h [n_elem, dim], elem_face [n_elem, 2*dim] (int64),
    face_elem [n_face, 2] (int64), face_local [n_face, 2] (int8),
    face_tag [n_face] (int32).
    """
    n = [int(v) for v in n]
    dim = len(n)
    assert dim in (2, 3)
    lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.ones(dim) if hi is None else np.asarray(hi, dtype=np.float64)
    h = (hi - lo) / np.asarray(n, dtype=np.float64)

    n_elem = int(np.prod(n))
    idx = np.indices(n[::-1]).reshape(dim, -1)[::-1]  # idx[a][e] = i_a, axis 0 fastest
    elem_lo = np.empty((n_elem, dim))
    elem_h = np.empty((n_elem, dim))
    for a in range(dim):
        elem_lo[:, a] = lo[a] + idx[a] * h[a]
        elem_h[:, a] = h[a]

    strides = [1, n[0], n[0] * (n[1] if dim > 1 else 1)]

    def eid(ii):
        return sum(int(ii[a]) * strides[a] for a in range(dim))

    elem_face = np.full((n_elem, 2 * dim), -1, dtype=np.int64)
    face_elem = []
    face_local = []
    face_tag = []
    fid = 0
    for ax in range(dim):
        shape = [n[a] + (1 if a == ax else 0) for a in range(dim)]
        grid = np.indices(shape[::-1]).reshape(dim, -1)[::-1]
        for col in range(grid.shape[1]):
            ii = [int(grid[a][col]) for a in range(dim)]
            k = ii[ax]
            if 0 < k < n[ax]:
                lo_e = list(ii)
                lo_e[ax] = k - 1
                em, ep = eid(lo_e), eid(ii)
                face_elem.append((em, ep))
                face_local.append((2 * ax + 1, 2 * ax))
                face_tag.append(TAG_INTERIOR)
                elem_face[em, 2 * ax + 1] = fid
                elem_face[ep, 2 * ax] = fid
            elif k == 0:
                em = eid(ii)
                face_elem.append((em, -1))
                face_local.append((2 * ax, -1))
                face_tag.append(boundary_tag)
                elem_face[em, 2 * ax] = fid
            else:
                lo_e = list(ii)
                lo_e[ax] = k - 1
                em = eid(lo_e)
                face_elem.append((em, -1))
                face_local.append((2 * ax + 1, -1))
                face_tag.append(boundary_tag)
                elem_face[em, 2 * ax + 1] = fid
            fid += 1
    return dict(
        dim=dim,
        n_elem=n_elem,
        n_face=fid,
        elem_lo=elem_lo,
        elem_h=elem_h,
        elem_face=elem_face,
        face_elem=np.asarray(face_elem, dtype=np.int64),
        face_local=np.asarray(face_local, dtype=np.int8),
        face_tag=np.asarray(face_tag, dtype=np.int32),
    )


# ---------------------------------------------------------------------------
# analytic fields (evaluated at caller-supplied coordinates x[..., dim])
# ---------------------------------------------------------------------------

def gaussian(x, center, sigma, amp=1.0):
    """amp * exp(-|x - c|^2 / (2 sigma^2))."""
    d = x - np.asarray(center, dtype=np.float64)
    return amp * np.exp(-np.sum(d * d, axis=-1) / (2.0 * sigma * sigma))


@dataclass
class FourierPerturbation:
    """Sum of M cosine modes per velocity component, amplitude a/M each."""
    k: np.ndarray          # [dim, M, dim] integer wave vectors
    theta: np.ndarray      # [dim, M] phases
    amp: float

    def __call__(self, x):
        dim = x.shape[-1]
        m = self.k.shape[1]
        out = np.zeros(x.shape[:-1] + (dim,))
        for c in range(dim):
            for j in range(m):
                arg = 2.0 * math.pi * (x @ self.k[c, j].astype(np.float64)) + self.theta[c, j]
                out[..., c] += (self.amp / m) * np.cos(arg)
        return out


@dataclass
class Workload:
    """One synthetic problem: mesh, PDE coefficients, initial and boundary data."""
    name: str
    pde: str                      # "transport" | "sw"
    dim: int
    n: tuple
    p: int
    scheme: str                   # "be" | "cn" | "steady"
    dt: float
    n_steps: int
    tol: float
    beta_const: np.ndarray | None = None
    beta_fn: object = None        # callable x -> beta(x) [..., dim] (variable case)
    Phi: float = 1.0
    u0_fn: object = None          # callable x -> u0 (transport) or (phi, u, v) for sw
    g_fn: object = None           # callable (x, t) -> boundary value (transport)
    f_fn: object = None           # callable x -> forcing at volume nodes (transport), or None
    noise_amp: float = 0.0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    def mesh(self):
        tag = TAG_WALL if self.pde == "sw" else TAG_DIRICHLET
        return structured_mesh(self.n, boundary_tag=tag)

    def noise(self, n_elem, n_nodes):
        """Seeded U(-a, a) per volume node, shape [n_elem, n_nodes]."""
        rng = np.random.default_rng(self.seed + 7919)
        return rng.uniform(-self.noise_amp, self.noise_amp, size=(n_elem, n_nodes))

    def initial(self, x_nodes):
        """Initial nodal values given node coordinates x_nodes [n_elem, Np, dim].

        Transport: [n_elem, 1, Np]; shallow water: [n_elem, 3, Np]."""
        n_elem, n_nodes, _ = x_nodes.shape
        if self.pde == "sw":
            out = np.zeros((n_elem, 3, n_nodes))
            out[:, 0, :] = self.u0_fn(x_nodes)
            return out
        u = self.u0_fn(x_nodes)
        if self.noise_amp > 0.0:
            u = u + self.noise(n_elem, n_nodes)
        return u[:, None, :]

    def beta_nodes(self, x_nodes):
        """Nodal velocity [n_elem, dim, Np] (variable-beta workloads only)."""
        b = self.beta_fn(x_nodes)  # [n_elem, Np, dim]
        return np.ascontiguousarray(np.transpose(b, (0, 2, 1)))

    def forcing(self, x_nodes):
        """Forcing at the volume nodes [n_elem, 1, Np], or None."""
        if self.f_fn is None:
            return None
        return self.f_fn(x_nodes)[:, None, :]

    def boundary(self, x_face_nodes, t):
        """Boundary data at face nodes x_face_nodes [n_face, Nfp, dim] at time t."""
        if self.g_fn is None:
            return np.zeros(x_face_nodes.shape[:-1])
        return self.g_fn(x_face_nodes, t)


def _advected_gaussian(beta, center, sigma):
    beta = np.asarray(beta, dtype=np.float64)

    def g(x, t):
        return gaussian(x - beta * t, center, sigma)

    return g


def transport_2d_small(n=(16, 16), p=2, dt=0.01, n_steps=10, tol=1e-10, seed=1001):
    """2D transport, constant beta = (1, 0.5), Gaussian bump at (0.3, 0.3),
    sigma 0.1, plus U(+-1e-3) noise; backward Euler."""
    beta = np.array([1.0, 0.5])
    c, s = (0.3, 0.3), 0.1
    return Workload(
        name=f"transport2d_{n[0]}x{n[1]}_p{p}_be", pde="transport", dim=2, n=tuple(n), p=p,
        scheme="be", dt=dt, n_steps=n_steps, tol=tol, beta_const=beta,
        u0_fn=lambda x: gaussian(x, c, s), g_fn=_advected_gaussian(beta, c, s),
        noise_amp=1e-3, seed=seed)


def variable_beta_field(seed=1002, n_modes=8, amp=0.05):
    """beta(x, y) = 0.5 (cos 2 pi y, sin 2 pi x) + Fourier perturbation."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 5, size=(2, n_modes, 2))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=(2, n_modes))
    pert = FourierPerturbation(k=k, theta=theta, amp=amp)

    def beta(x):
        out = np.empty(x.shape)
        out[..., 0] = 0.5 * np.cos(2.0 * math.pi * x[..., 1])
        out[..., 1] = 0.5 * np.sin(2.0 * math.pi * x[..., 0])
        return out + pert(x)

    return beta


def transport_2d_variable(n=(256, 256), p=4, dt=2e-3, n_steps=50, tol=1e-10, seed=1002):
    """2D transport with per-element velocity (smooth field plus 8 random
    Fourier modes of amplitude 0.05), Crank-Nicolson; inflow data frozen in time
    (the smooth part of the initial condition)."""
    c, s = (0.3, 0.3), 0.1
    return Workload(
        name=f"transport2d_varbeta_{n[0]}x{n[1]}_p{p}_cn", pde="transport", dim=2, n=tuple(n),
        p=p, scheme="cn", dt=dt, n_steps=n_steps, tol=tol,
        beta_fn=variable_beta_field(seed), u0_fn=lambda x: gaussian(x, c, s),
        g_fn=lambda x, t: gaussian(x, c, s), noise_amp=1e-3, seed=seed)


def steady_2d_smooth(n=(256, 256), p=4, tol=1e-10):
    """Steady 2D transport with the smooth solution of the paper's first
    experiment (Sec. 4.1): beta = (y, x) on the unit square, u_e =
    sin(pi x) cos(pi y) / pi, forcing f = beta . grad u_e, inflow data u_e,
    zero initial guess. Per-node velocity, so per-element operators."""
    def ue(x):
        return np.sin(math.pi * x[..., 0]) * np.cos(math.pi * x[..., 1]) / math.pi

    def fe(x):
        return (x[..., 1] * np.cos(math.pi * x[..., 0]) * np.cos(math.pi * x[..., 1])
                - x[..., 0] * np.sin(math.pi * x[..., 0]) * np.sin(math.pi * x[..., 1]))

    return Workload(
        name=f"steady2d_smooth_{n[0]}x{n[1]}_p{p}", pde="transport", dim=2, n=tuple(n), p=p,
        scheme="steady", dt=1.0, n_steps=1, tol=tol,
        beta_fn=lambda x: np.stack([x[..., 1], x[..., 0]], -1),
        u0_fn=lambda x: np.zeros(x.shape[:-1]), g_fn=lambda x, t: ue(x), f_fn=fe,
        meta={"exact": ue})


def sw_2d(n=(512, 512), p=3, dt=1e-3, n_steps=100, tol=1e-10, seed=1003, n_bumps=16):
    """Linearised shallow water, Phi = 1, walls; height = random-phase sum of
    Gaussian bumps, zero velocity; backward Euler."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.1, 0.9, size=(n_bumps, 2))
    sigmas = rng.uniform(0.02, 0.08, size=n_bumps)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=n_bumps)

    def phi0(x):
        out = np.zeros(x.shape[:-1])
        for m in range(n_bumps):
            out += math.cos(phases[m]) * gaussian(x, centers[m], sigmas[m])
        return out

    return Workload(
        name=f"sw2d_{n[0]}x{n[1]}_p{p}_be", pde="sw", dim=2, n=tuple(n), p=p, scheme="be",
        dt=dt, n_steps=n_steps, tol=tol, Phi=1.0, u0_fn=phi0, seed=seed)


def transport_3d(n=(64, 64, 64), p=3, dt=5e-3, n_steps=20, tol=1e-10, seed=1004):
    """3D transport, beta = (1,1,1)/sqrt(3), Gaussian at (0.3,0.3,0.3) with
    sigma 0.08 plus U(+-1e-3) noise; backward Euler."""
    beta = np.ones(3) / math.sqrt(3.0)
    c, s = (0.3, 0.3, 0.3), 0.08
    return Workload(
        name=f"transport3d_{n[0]}x{n[1]}x{n[2]}_p{p}_be", pde="transport", dim=3, n=tuple(n),
        p=p, scheme="be", dt=dt, n_steps=n_steps, tol=tol, beta_const=beta,
        u0_fn=lambda x: gaussian(x, c, s), g_fn=_advected_gaussian(beta, c, s),
        noise_amp=1e-3, seed=seed)


def batched_mix(n_inst=256, seed=1005, n_range=(8, 128), p_range=(1, 5)):
    """Independent 2D transport instances: side N = round(8 * 16^U) (log-uniform
    in 8..128), p uniform in 1..5, constant beta = s (cos t, sin t) with
    s ~ U(0.5, 1.5), Gaussian initial data with random centre and width."""
    rng = np.random.default_rng(seed)
    out = []
    lo_n, hi_n = n_range
    for i in range(n_inst):
        nn = int(round(lo_n * (hi_n / lo_n) ** rng.uniform()))
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        th = rng.uniform(0.0, 2.0 * math.pi)
        sp = rng.uniform(0.5, 1.5)
        beta = sp * np.array([math.cos(th), math.sin(th)])
        c = rng.uniform(0.2, 0.8, size=2)
        s = rng.uniform(0.05, 0.15)
        out.append(Workload(
            name=f"inst{i}_{nn}x{nn}_p{p}", pde="transport", dim=2, n=(nn, nn), p=p,
            scheme="be", dt=0.01, n_steps=10, tol=1e-10, beta_const=beta,
            u0_fn=(lambda x, c=c, s=s: gaussian(x, c, s)),
            g_fn=_advected_gaussian(beta, c, s), seed=seed + i))
    return out
