"""1D polynomial machinery (test infrastructure only; see oracle/__init__.py).

The paper fixes neither basis nor quadrature (Sec. 2 only asks for degree-p
polynomials per element and per face). Readings used throughout the oracle:
  * tensor-product Lagrange basis on the p+1 Gauss-Lobatto-Legendre (GLL)
    points of [-1, 1] per axis (the Q^p space, since every mesh in Sec. 4 is
    made of quads/hexes); for p = 0 the one node is the centre (nodes_1d);
  * Gauss-Legendre quadrature with enough points to integrate every product
    exactly (q = p+1 for constant coefficients, ceil(3p/2)+1 when the velocity
    is a degree-p interpolant).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gll(p):
    """GLL nodes and weights on [-1, 1] for degree p >= 1.

    Nodes: -1, 1 and the roots of P_p'. Weights: 2 / (p (p+1) P_p(x)^2).
    """
    if p < 1:
        raise ValueError("GLL needs p >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    inner = np.real(npleg.legroots(npleg.legder(cp))) if p > 1 else np.zeros(0)
    # polish the interior roots with Newton on P_p'
    d1 = npleg.legder(cp)
    d2 = npleg.legder(cp, 2)
    for _ in range(6):
        if inner.size:
            inner = inner - npleg.legval(inner, d1) / npleg.legval(inner, d2)
    x = np.concatenate(([-1.0], np.sort(inner), [1.0]))
    w = 2.0 / (p * (p + 1) * npleg.legval(x, cp) ** 2)
    return x, w


def nodes_1d(p):
    """Nodes and weights of the 1D nodal basis of degree p: the GLL points for
    p >= 1; for p = 0 (the piecewise-constant space of Sec. 2 with p = 0) the
    single node at the centre of [-1, 1], weight 2."""
    if p == 0:
        return np.zeros(1), np.full(1, 2.0)
    return gll(p)


def gauss(q):
    """Gauss-Legendre rule with q points on [-1, 1] (numpy's leggauss)."""
    return npleg.leggauss(q)


def lagrange(nodes, x):
    """L[g, a] = l_a(x_g) for the Lagrange basis on `nodes`."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    L = np.ones((x.size, n))
    for a in range(n):
        for b in range(n):
            if b != a:
                L[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return L


def lagrange_deriv(nodes, x):
    """D[g, a] = l_a'(x_g), by the product rule on the Lagrange product."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    D = np.zeros((x.size, n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[m]))
            for b in range(n):
                if b != a and b != m:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            D[:, a] += term
    return D


def quad_points(p, variable_coeff):
    """Number of Gauss points per axis: p+1, or ceil(3p/2)+1 for a degree-p
    coefficient inside the integrand."""
    return (3 * p + 1) // 2 + 1 if variable_coeff else p + 1


def mass_1d(p, q=None):
    """M1[a, b] = int l_a l_b on [-1, 1] (row = test function)."""
    r, _ = gll(p)
    xi, om = gauss(q or p + 1)
    L = lagrange(r, xi)
    return L.T @ (om[:, None] * L)


def stiff_1d(p, q=None):
    """S1[a, b] = int l_a' l_b on [-1, 1] (row = test function derivative)."""
    r, _ = gll(p)
    xi, om = gauss(q or p + 1)
    L = lagrange(r, xi)
    D = lagrange_deriv(r, xi)
    return D.T @ (om[:, None] * L)
