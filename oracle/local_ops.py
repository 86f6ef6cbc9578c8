"""Element operators of the upwind HDG local equations (test infrastructure only).

For one axis-aligned element K with corner lo and edge lengths h, everything is
integrated with Gauss quadrature on the reference box (x = lo + h (r+1)/2,
volume Jacobian J = prod h/2, face Jacobian J_f = prod over tangential h/2).

Transport (Sec. 3, eq. transportLocal, with the time term of Sec. 3's
time-dependent paragraph): for trial u and test v in Q^p(K)
    A_sp(u, v) = -(u, div(beta v))_K + <(beta.n + |beta.n|) u, v>_dK
    B(uhat, v) = <|beta.n| uhat, v>_dK
so that the local equation reads  A_sp u - B uhat = (f, v)_K  (steady) and
(u/dt, v)_K + A_sp u - B uhat = (f + u^n/dt, v)_K  (backward Euler).

Shallow water (Sec. 3, eq. localSolverDD, f = gamma = tau = 0), unknowns
(phi, u, v), scalar trace phihat:
    phi-row: -(Phi vel, grad w)_K + <Phi vel.n + sqrt(Phi) phi, w>_dK  -  sqrt(Phi) <phihat, w>_dK
    u-row:   -(Phi phi, dw/dx)_K                                      +  Phi <phihat n_x, w>_dK
    v-row:   -(Phi phi, dw/dy)_K                                      +  Phi <phihat n_y, w>_dK
with the time term blockdiag(1, Phi, Phi) (., w)_K / dt.

Readings: beta enters as its degree-p GLL interpolant on each element (the
variable-velocity workload), integrated exactly with ceil(3p/2)+1 Gauss points;
constant beta uses p+1 points (exact as well). The trace uhat appears only
inside the face integrals, so it is represented by its values at the face
Gauss points (the same rule as the volume, restricted to the face): B maps
those point values to the right-hand side. The trace formula of the
iteration is evaluated at exactly these points.
"""
from __future__ import annotations

import numpy as np

from .basis import gauss, lagrange, lagrange_deriv, nodes_1d, quad_points


def _tensor(mats):
    """Tensor product of 1D evaluation matrices mats[a] of shape [q_a, n_a].

    Returns [prod q_a, prod n_a] with axis 0 fastest in both index spaces."""
    out = mats[0]
    for m in mats[1:]:
        # new index: (old) + size_old * (new axis)
        out = np.einsum("ga,hb->hgba", out, m).reshape(out.shape[0] * m.shape[0],
                                                         out.shape[1] * m.shape[1])
    return out


class RefElement:
    """Reference-element tables for dimension dim, degree p, q Gauss points."""

    def __init__(self, dim, p, q):
        self.dim, self.p, self.q = dim, p, q
        self.r, self.wgll = nodes_1d(p)
        self.xi, self.om = gauss(q)
        L = lagrange(self.r, self.xi)
        D = lagrange_deriv(self.r, self.xi)
        self.Np = (p + 1) ** dim
        self.Nfp = (p + 1) ** (dim - 1)
        self.Nqf = q ** (dim - 1)                          # trace points per face
        # volume tables
        self.phi = _tensor([L] * dim)                      # [Q, Np]
        self.dphi = []
        for ax in range(dim):
            mats = [D if a == ax else L for a in range(dim)]
            self.dphi.append(_tensor(mats))                # reference d/dr_ax
        self.W = _tensor([self.om[:, None]] * dim)[:, 0]   # [Q]
        # reference coordinates of the volume points (axis 0 fastest, as in _tensor)
        idx = np.indices((q,) * dim).reshape(dim, -1)[::-1]
        self.X = np.stack([self.xi[idx[a]] for a in range(dim)], -1)   # [Q, dim]
        # face tables, local face f = 2*ax + side
        self.fphi, self.fpsi, self.fW = [], [], []
        for f in range(2 * dim):
            ax, side = divmod(f, 2)
            end = lagrange(self.r, [1.0 if side else -1.0])  # [1, p+1]
            mats = [end if a == ax else L for a in range(dim)]
            self.fphi.append(_tensor(mats))                # [Qf, Np]
            tang = [L for a in range(dim) if a != ax]
            self.fpsi.append(_tensor(tang) if tang else np.ones((1, 1)))
            wt = [self.om[:, None] for a in range(dim) if a != ax]
            self.fW.append(_tensor(wt)[:, 0] if wt else np.ones(1))


def _geometry(h):
    h = np.asarray(h, dtype=np.float64)
    J = np.prod(h / 2.0)
    Jf = [J * 2.0 / h[ax] for ax in range(h.size)]
    return J, Jf


def transport_element(ref, h, beta_nodes):
    """(M, A_sp, B) for one transport element.

    beta_nodes: [dim, Np] nodal velocity (a constant velocity is passed as
    constant nodal values). B has columns ordered (local face f, face point g).
    """
    dim, Np = ref.dim, ref.Np
    J, Jf = _geometry(h)
    h = np.asarray(h, dtype=np.float64)
    W = ref.W * J
    M = ref.phi.T @ (W[:, None] * ref.phi)

    bq = [ref.phi @ beta_nodes[ax] for ax in range(dim)]          # beta_ax at points
    dbq = [ref.dphi[ax] @ beta_nodes[ax] for ax in range(dim)]    # d beta_ax / d r_ax
    # div(beta phi_i) at quadrature points, [Q, Np]
    div = np.zeros_like(ref.phi)
    for ax in range(dim):
        div += (2.0 / h[ax]) * (dbq[ax][:, None] * ref.phi + bq[ax][:, None] * ref.dphi[ax])
    # -(phi_j, div(beta phi_i)) : row i, column j
    Asp = -(div.T @ (W[:, None] * ref.phi))

    Nqf = ref.Nqf
    B = np.zeros((Np, 2 * dim * Nqf))
    for f in range(2 * dim):
        ax, side = divmod(f, 2)
        sgn = 1.0 if side else -1.0
        Phi_f = ref.fphi[f]
        bn = sgn * (Phi_f @ beta_nodes[ax])                       # beta.n at face points
        wf = ref.fW[f] * Jf[ax]
        Asp += Phi_f.T @ ((wf * (bn + np.abs(bn)))[:, None] * Phi_f)
        B[:, f * Nqf:(f + 1) * Nqf] = Phi_f.T * (wf * np.abs(bn))[None, :]
    return M, Asp, B


def sw_element(ref, h, Phi, lo=None, coriolis=(0.0, 0.0, 0.0), friction=0.0):
    """(Mblk, A_sp, B) for one 2D linearised shallow-water element.

    Unknown order (phi, u, v), each Np nodal values; B maps the scalar trace
    phihat (ordered by local face, face point) to the three right-hand sides.
    Source terms of eq. linearizedShallow, moved to the left-hand side of the
    local equations (Sec. 3, eq. localSolverDD): bottom friction gamma adds
    (gamma Phi u, w) to the u-row and (gamma Phi v, w) to the v-row; the
    Coriolis parameter f = f0 + beta (y - y_m) adds -(f Phi v, w) to the
    u-row and +(f Phi u, w) to the v-row, with f at the volume quadrature
    points of the element whose lower corner is lo. coriolis = (f0, beta, y_m)."""
    assert ref.dim == 2
    Np = ref.Np
    J, Jf = _geometry(h)
    h = np.asarray(h, dtype=np.float64)
    W = ref.W * J
    M = ref.phi.T @ (W[:, None] * ref.phi)
    f0, beta_c, y_m = (float(v) for v in coriolis)
    gamma = float(friction)
    sq = np.sqrt(Phi)
    # G_ax[i, j] = (phi_j, d phi_i / dx_ax)_K
    G = [(2.0 / h[ax]) * (ref.dphi[ax].T @ (W[:, None] * ref.phi)) for ax in range(2)]
    n = 3 * Np
    A = np.zeros((n, n))
    A[0:Np, Np:2 * Np] = -Phi * G[0]
    A[0:Np, 2 * Np:3 * Np] = -Phi * G[1]
    A[Np:2 * Np, 0:Np] = -Phi * G[0]
    A[2 * Np:3 * Np, 0:Np] = -Phi * G[1]
    Nqf = ref.Nqf
    B = np.zeros((n, 4 * Nqf))
    for f in range(4):
        ax, side = divmod(f, 2)
        nrm = np.zeros(2)
        nrm[ax] = 1.0 if side else -1.0
        Phi_f = ref.fphi[f]
        wf = ref.fW[f] * Jf[ax]
        Ef = Phi_f.T @ (wf[:, None] * Phi_f)            # face mass on volume basis
        Bf = Phi_f.T * wf[None, :]                       # volume test x trace point value
        A[0:Np, 0:Np] += sq * Ef
        A[0:Np, Np:2 * Np] += Phi * nrm[0] * Ef
        A[0:Np, 2 * Np:3 * Np] += Phi * nrm[1] * Ef
        cols = slice(f * Nqf, (f + 1) * Nqf)
        B[0:Np, cols] = sq * Bf
        B[Np:2 * Np, cols] = -Phi * nrm[0] * Bf
        B[2 * Np:3 * Np, cols] = -Phi * nrm[1] * Bf
    if gamma != 0.0:
        A[Np:2 * Np, Np:2 * Np] += gamma * Phi * M
        A[2 * Np:3 * Np, 2 * Np:3 * Np] += gamma * Phi * M
    if f0 != 0.0 or beta_c != 0.0:
        lo_y = 0.0 if lo is None else float(np.asarray(lo)[1])
        y_q = lo_y + 0.5 * h[1] * (ref.X[:, 1] + 1.0)     # physical y of the quadrature points
        fq = f0 + beta_c * (y_q - y_m)
        Mf = ref.phi.T @ ((W * fq)[:, None] * ref.phi)
        A[Np:2 * Np, 2 * Np:3 * Np] -= Phi * Mf
        A[2 * Np:3 * Np, Np:2 * Np] += Phi * Mf
    Mblk = np.zeros((n, n))
    Mblk[0:Np, 0:Np] = M
    Mblk[Np:2 * Np, Np:2 * Np] = Phi * M
    Mblk[2 * Np:3 * Np, 2 * Np:3 * Np] = Phi * M
    return Mblk, A, B


def make_ref(dim, p, variable_beta):
    return RefElement(dim, p, quad_points(p, variable_beta))
