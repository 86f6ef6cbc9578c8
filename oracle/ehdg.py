"""The eHDG iteration, Algorithm 1 of the paper (test infrastructure only).

One implicit time step (or one steady solve) runs Algorithm 1:
  given the initial guess u^0, compute the initial trace uhat^0 with the trace
  formula; then repeat { solve every element's local equation for u^{k+1}
  with the trace uhat^k (eq. transportLocalk1 / localSolverDD); compute
  uhat^{k+1} with the trace formula (eq. transportLocale / the shallow-water
  trace of Sec. 3); check convergence }.

Readings (the paper leaves these open):
  * Jacobi order: every element uses uhat^k, every face uses u^{k+1}.
  * Warm start: u^0 of a time step is the previous step's solution (Sec. 4.4:
    the initial guess of each step is the previous step's solution); the
    initial trace is the trace formula applied to it with the new step's
    boundary data.
  * Convergence: r_k = || uhat^{k+1} - uhat^k ||_{L2(E_h)} < tol, the L2 norm on
    the skeleton evaluated with the face Gauss rule; r_k is recorded every
    iteration. Steady solves start from u^0 = 0.
  * The trace formula is evaluated pointwise at the face quadrature points,
    the only places where the local equations use the trace; sgn(0) = 0 as
    written. (Evaluating it at face GLL nodes instead and interpolating breaks
    the iteration at stagnation nodes: for beta = (y, x) of Sec. 4.1 the
    iteration then diverges at p = 4.) Transport boundary: the formula with the exterior value u^+ = g
    (so uhat = g on inflow nodes, u^- on outflow nodes). Shallow-water wall: the
    formula with the mirror state phi^+ = phi^-, vel^+.n^+ = vel^-.n^-, i.e.
    phihat = phi^- + sqrt(Phi) vel^-.n^-. The sign of beta.n at a face node is
    taken from the minus element's nodal velocity.
  * Crank-Nicolson (time discretisation not in the paper, textbook form):
    (M/dt)(u^{n+1}-u^n) + 1/2 [a(u^{n+1}, uhat^{n+1}) + a(u^n, uhat^n)]
    = 1/2 (F^{n+1} + F^n), where a(u, uhat) = A_sp u - B uhat, with uhat^n the
    previous step's converged trace (at the first step, the trace formula of
    u^0 with the boundary data at t = 0).
  * Forcing is given as nodal values of the right-hand side of the evolution
    equations (transport: u_t + beta.grad u = f; shallow water:
    phi_t + Phi div vel = f_phi, vel_t + grad phi = f_vel), entering as
    blockdiag(1, Phi, Phi) M f.
"""
from __future__ import annotations

import numpy as np

from . import local_ops
from .geometry import face_volume_nodes


class Problem:
    """Mesh + PDE + element operators. mesh is the dict of connectivity arrays
    (elements, faces, face_elem/face_local/elem_face, face_tag)."""

    def __init__(self, mesh, p, pde="transport", scheme="be", dt=1.0, Phi=1.0,
                 beta_const=None, beta_nodes=None, coriolis=(0.0, 0.0, 0.0), friction=0.0):
        self.mesh = mesh
        self.p, self.pde, self.scheme, self.dt, self.Phi = p, pde, scheme, float(dt), float(Phi)
        self.dim = dim = mesh["dim"]
        self.nel, self.nface = mesh["n_elem"], mesh["n_face"]
        variable = beta_nodes is not None
        # shallow water: Coriolis f = f0 + beta (y - y_m) and bottom friction
        # gamma (eq. linearizedShallow); a beta-plane makes every element's
        # operator different
        self.coriolis = tuple(float(v) for v in coriolis)
        self.friction = float(friction)
        sw_varying = pde == "sw" and self.coriolis[1] != 0.0
        self.ref = ref = local_ops.make_ref(dim, p, variable)
        self.Np, self.Nfp = ref.Np, ref.Nfp
        self.nf = 3 if pde == "sw" else 1
        self.n = self.nf * self.Np
        self.fvn = [face_volume_nodes(dim, p, f) for f in range(2 * dim)]
        h = mesh["elem_h"]
        uniform = np.allclose(h, h[0], rtol=0, atol=0)
        if pde == "transport":
            if variable:
                self.beta_nodes = np.asarray(beta_nodes, dtype=np.float64)
            else:
                bc = np.asarray(beta_const, dtype=np.float64)
                self.beta_nodes = np.broadcast_to(bc[None, :, None], (self.nel, dim, self.Np))
        else:
            self.beta_nodes = None
        if (not variable) and (not sw_varying) and uniform:
            ops = self._element_ops(0)
            self.M, self.Asp, self.B = (np.broadcast_to(o, (self.nel,) + o.shape) for o in ops)
        else:
            ops = [self._element_ops(e) for e in range(self.nel)]
            self.M = np.stack([o[0] for o in ops])
            self.Asp = np.stack([o[1] for o in ops])
            self.B = np.stack([o[2] for o in ops])
        # quadrature weights of the skeleton L2 norm (face Gauss rule times J_f)
        self.Nqf = ref.Nqf
        self.face_w = np.empty((self.nface, ref.Nqf))
        for e in range(self.nface):
            em, fm = mesh["face_elem"][e, 0], int(mesh["face_local"][e, 0])
            hh = h[em]
            self.face_w[e] = ref.fW[fm] * np.prod(hh / 2.0) * 2.0 / hh[fm // 2]

    def _element_ops(self, e):
        h = self.mesh["elem_h"][e]
        if self.pde == "transport":
            return local_ops.transport_element(self.ref, h, self.beta_nodes[e])
        return local_ops.sw_element(self.ref, h, self.Phi, lo=self.mesh["elem_lo"][e],
                                    coriolis=self.coriolis, friction=self.friction)

    # -- the trace formula ---------------------------------------------------
    def face_values(self, u, e, side):
        """Values of every field of u at the quadrature points of face e, seen
        from its minus (0) or plus (1) element: ([nf, Nqf], local face)."""
        el = self.mesh["face_elem"][e, side]
        f = int(self.mesh["face_local"][e, side])
        return u[el] @ self.ref.fphi[f].T, f

    def beta_normal(self, e):
        """beta.n^- at the quadrature points of face e, from the minus element."""
        em, fm = self.mesh["face_elem"][e, 0], int(self.mesh["face_local"][e, 0])
        ax, side = divmod(fm, 2)
        nsgn = 1.0 if side else -1.0
        return nsgn * (self.ref.fphi[fm] @ self.beta_nodes[em, ax])

    def trace(self, u, g=None):
        """uhat at every face quadrature point, [nface, Nqf], from the element
        values u [nel, nf, Np] (eq. transportLocale, or the shallow-water trace
        of Sec. 3). g: boundary data at the face points of boundary faces."""
        uh = np.empty((self.nface, self.ref.Nqf))
        sq = np.sqrt(self.Phi)
        for e in range(self.nface):
            vm, fm = self.face_values(u, e, 0)
            ax, side = divmod(fm, 2)
            nsgn = 1.0 if side else -1.0                        # n^- = nsgn e_ax
            interior = self.mesh["face_elem"][e, 1] >= 0
            if self.pde == "transport":
                s_m = np.sign(self.beta_normal(e))              # sgn(beta.n^-)
                s_p = -s_m                                      # n^+ = -n^-
                u_m = vm[0]
                u_p = self.face_values(u, e, 1)[0][0] if interior else g[e]
                uh[e] = 0.5 * (u_m * s_m + u_p * s_p) + 0.5 * (u_m + u_p)
            else:
                phi_m, un_m = vm[0], nsgn * vm[1 + ax]           # vel^-.n^-
                if interior:
                    vp, _ = self.face_values(u, e, 1)
                    phi_p, un_p = vp[0], -nsgn * vp[1 + ax]      # vel^+.n^+
                else:
                    phi_p, un_p = phi_m, un_m                    # mirror state at a wall
                uh[e] = 0.5 * (phi_m + phi_p) + sq * 0.5 * (un_m + un_p)
        return uh

    def trace_norm(self, duh):
        """|| duh ||_{L2(E_h)} with the face Gauss rule."""
        return float(np.sqrt(np.sum(self.face_w * duh * duh)))

    def gather(self, uh):
        """Per-element stack of its faces' traces, [nel, 2d*Nqf] (local face order)."""
        return uh[self.mesh["elem_face"]].reshape(self.nel, -1)

    # -- one implicit step ---------------------------------------------------
    def _mass(self):
        if self.pde == "transport":
            return self.M
        return self.M  # sw_element already returns blockdiag(M, Phi M, Phi M)

    def step_system(self, u_n, uh_n, f_new=None, f_old=None):
        """(A, r0, cB): the local systems A u^{k+1} = r0 + cB B uhat^k of one step."""
        M, Asp, B = self._mass(), self.Asp, self.B
        un = u_n.reshape(self.nel, self.n)
        fn = None if f_new is None else f_new.reshape(self.nel, self.n)
        fo = None if f_old is None else f_old.reshape(self.nel, self.n)
        mv = lambda A, x: np.einsum("eij,ej->ei", A, x)
        dt = self.dt
        if self.scheme == "be":
            A = M / dt + Asp
            r0 = mv(M, un) / dt
            if fn is not None:
                r0 = r0 + mv(M, fn)
            return A, r0, 1.0
        if self.scheme == "cn":
            A = M / dt + 0.5 * Asp
            r0 = mv(M, un) / dt - 0.5 * mv(Asp, un) + 0.5 * mv(B, self.gather(uh_n))
            if fn is not None:
                r0 = r0 + 0.5 * mv(M, fn)
            if fo is not None:
                r0 = r0 + 0.5 * mv(M, fo)
            return A, r0, 0.5
        if self.scheme == "steady":
            r0 = np.zeros((self.nel, self.n)) if fn is None else mv(M, fn)
            return Asp, r0, 1.0
        raise ValueError(self.scheme)

    def solve_step(self, u_n, uh_n=None, g_new=None, f_new=None, f_old=None, tol=1e-10,
                   max_iter=1000, fixed_iters=None, u_init=None, stop=None):
        """Algorithm 1 for one implicit step (or the steady problem).

        Returns (u, uhat, history) with u [nel, nf, Np], uhat [nface, Nqf] and
        history the list of r_k. fixed_iters runs exactly that many iterations;
        stop(u_new, u_old) -> bool replaces the trace-increment test."""
        A, r0, cB = self.step_system(u_n, uh_n, f_new, f_old)
        u = (u_n if u_init is None else u_init).reshape(self.nel, self.nf, self.Np).copy()
        uh = self.trace(u, g_new)
        hist = []
        n_it = fixed_iters if fixed_iters is not None else max_iter
        for _ in range(n_it):
            rhs = r0 + cB * np.einsum("eij,ej->ei", self.B, self.gather(uh))
            u_new = np.linalg.solve(A, rhs[..., None])[..., 0].reshape(self.nel, self.nf, self.Np)
            uh_new = self.trace(u_new, g_new)
            r = self.trace_norm(uh_new - uh)
            hist.append(r)
            done = (stop(u_new, u) if stop is not None else r < tol)
            u, uh = u_new, uh_new
            if fixed_iters is None and done:
                break
        return u, uh, hist

    def run(self, u0, n_steps, g_of_t=None, f_of_t=None, tol=1e-10, max_iter=1000,
            fixed_iters=None):
        """n_steps implicit steps from u0; g_of_t(t) -> boundary data [nface, Nqf],
        f_of_t(t) -> forcing [nel, nf, Np]. Returns (u, uhat, iterations per
        step, residual histories)."""
        u = u0.reshape(self.nel, self.nf, self.Np).copy()
        g = (lambda t: None) if g_of_t is None else g_of_t
        f = (lambda t: None) if f_of_t is None else f_of_t
        uh = self.trace(u, g(0.0))
        iters, hists = [], []
        for n in range(n_steps):
            t_old, t_new = n * self.dt, (n + 1) * self.dt
            u, uh, hist = self.solve_step(u, uh, g(t_new), f(t_new), f(t_old), tol=tol,
                                          max_iter=max_iter, fixed_iters=fixed_iters)
            iters.append(len(hist))
            hists.append(hist)
        return u, uh, iters, hists


def l2_volume(prob, u, exact=None, extra_q=3):
    """|| u_h - exact ||_{L2(Omega)} for field 0 (or || u_h || if exact is None),
    with a (p+extra_q)-point Gauss rule per axis."""
    from .basis import gauss, lagrange
    from .local_ops import _tensor
    xi, om = gauss(prob.p + extra_q)
    Phi = _tensor([lagrange(prob.ref.r, xi)] * prob.dim)   # [Q, Np]
    W = _tensor([om[:, None]] * prob.dim)[:, 0]
    nq = xi.size
    pts = np.zeros((nq ** prob.dim, prob.dim))           # reference points, axis 0 fastest
    for g in range(nq ** prob.dim):
        rem = g
        for a in range(prob.dim):
            pts[g, a] = xi[rem % nq]
            rem //= nq
    lo, h = prob.mesh["elem_lo"], prob.mesh["elem_h"]
    vals = u.reshape(prob.nel, prob.nf, prob.Np)[:, 0, :] @ Phi.T   # [nel, Q]
    if exact is not None:
        x = lo[:, None, :] + h[:, None, :] * (pts[None, :, :] + 1.0) / 2.0
        vals = vals - exact(x)
    J = np.prod(h / 2.0, axis=1)
    return float(np.sqrt(np.sum(J[:, None] * W[None, :] * vals * vals)))
