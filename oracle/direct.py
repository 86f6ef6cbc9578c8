"""Direct solve of the monolithic upwind HDG system (test infrastructure only).

Unknowns: every element's volume values u_K and every face's trace uhat_e as a
polynomial in Q^p(e) (coefficients at the face GLL nodes). Rows:
  * the local equation of each element (Sec. 3, eq. transportLocal or
    localSolverDD), A_K u_K - cB B_K uhat_K = r0_K, with the same time
    discretisation as the iteration (oracle.ehdg.Problem.step_system);
  * the conservation condition on each face (Sec. 3: the jump of the upwind
    flux is orthogonal to every mu in Q^p(e)), integrated with the face Gauss
    rule:
      transport:  < (b + |b|) u^- + (|b| - b) u^+ - 2|b| uhat, mu >_e = 0,
                  b = beta.n^-, with u^+ = g on a boundary face;
      shallow water: < Phi (vel^-.n^- + vel^+.n^+) + sqrt(Phi)(phi^- + phi^+ - 2 phihat), mu >_e = 0,
                  and at a wall the zero-flux condition
                  < Phi vel^-.n^- + sqrt(Phi)(phi^- - phihat), mu >_e = 0.
Reading: where beta.n vanishes on a whole face the condition is void; the
trace there is the face average of the two sides (eq. transportLocale with
sgn(0) = 0). The sparse system is solved with scipy's LU.

This formulation differs from the iteration's (a weak, polynomial trace
instead of the pointwise trace formula), so agreement of the eHDG fixed point
with this solution is a genuine check of Algorithm 1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve(prob, u_n, uh_n=None, g=None, f_new=None, f_old=None):
    """Return (u [nel, nf, Np], uhat at the face points [nface, Nqf])."""
    mesh, ref = prob.mesh, prob.ref
    nel, n, nface, Nfp, Nqf = prob.nel, prob.n, prob.nface, prob.Nfp, ref.Nqf
    A, r0, cB = prob.step_system(u_n, uh_n, f_new, f_old)
    nu = nel * n
    N = nu + nface * Nfp
    rows, cols, vals = [], [], []
    rhs = np.zeros(N)

    def add(r, c, blk):
        rr, cc = np.meshgrid(np.atleast_1d(r), np.atleast_1d(c), indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(np.asarray(blk, dtype=np.float64).ravel())

    def tcols(e):
        return nu + e * Nfp + np.arange(Nfp)

    # element rows: the trace enters through its values at the face points
    for K in range(nel):
        ru = np.arange(K * n, (K + 1) * n)
        add(ru, ru, A[K])
        for f in range(2 * prob.dim):
            e = mesh["elem_face"][K, f]
            Bf = prob.B[K][:, f * Nqf:(f + 1) * Nqf]
            add(ru, tcols(e), -cB * (Bf @ ref.fpsi[f]))
        rhs[ru] = r0[K]

    sq = np.sqrt(prob.Phi)
    for e in range(nface):
        rf = tcols(e)
        em, fm = int(mesh["face_elem"][e, 0]), int(mesh["face_local"][e, 0])
        ep, fp = int(mesh["face_elem"][e, 1]), int(mesh["face_local"][e, 1])
        ax, side = divmod(fm, 2)
        nsgn = 1.0 if side else -1.0
        hh = mesh["elem_h"][em]
        w = ref.fW[fm] * np.prod(hh / 2.0) * 2.0 / hh[ax]
        psi = ref.fpsi[fm]                                    # [Nqf, Nfp]
        Pm = ref.fphi[fm]                                     # [Nqf, Np]
        Pp = ref.fphi[fp] if ep >= 0 else None
        Np = prob.Np
        if prob.pde == "transport":
            b = prob.beta_normal(e)
            ab = np.abs(b)
            if np.all(b == 0.0):
                if Nqf != Nfp:
                    raise NotImplementedError("face with beta.n = 0 everywhere, q != p+1")
                # average of the two sides, collocated at the face points
                add(rf, rf, psi)
                add(rf, em * n + np.arange(n), -0.5 * Pm)
                if ep >= 0:
                    add(rf, ep * n + np.arange(n), -0.5 * Pp)
                else:
                    rhs[rf] += 0.5 * g[e]
                continue
            add(rf, em * n + np.arange(n), psi.T @ ((w * (b + ab))[:, None] * Pm))
            add(rf, rf, -psi.T @ ((w * 2.0 * ab)[:, None] * psi))
            if ep >= 0:
                add(rf, ep * n + np.arange(n), psi.T @ ((w * (ab - b))[:, None] * Pp))
            else:
                rhs[rf] -= psi.T @ (w * (ab - b) * g[e])
        else:
            cm = np.zeros((Nqf, n))
            cm[:, 0:Np] = sq * Pm
            cm[:, (1 + ax) * Np:(2 + ax) * Np] = prob.Phi * nsgn * Pm
            add(rf, em * n + np.arange(n), psi.T @ (w[:, None] * cm))
            if ep >= 0:
                cp = np.zeros((Nqf, n))
                cp[:, 0:Np] = sq * Pp
                cp[:, (1 + ax) * Np:(2 + ax) * Np] = prob.Phi * (-nsgn) * Pp
                add(rf, ep * n + np.arange(n), psi.T @ (w[:, None] * cp))
                add(rf, rf, -psi.T @ ((w * 2.0 * sq)[:, None] * psi))
            else:
                add(rf, rf, -psi.T @ ((w * sq)[:, None] * psi))

    Aglob = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N))
    x = spla.spsolve(Aglob, rhs)
    uhp = x[nu:].reshape(nface, Nfp)
    uh_pts = np.stack([ref.fpsi[int(mesh["face_local"][e, 0])] @ uhp[e] for e in range(nface)])
    return x[:nu].reshape(nel, prob.nf, prob.Np), uh_pts
