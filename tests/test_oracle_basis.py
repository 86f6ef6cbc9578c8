"""Pins for the oracle's 1D machinery against closed forms (no GPU)."""
import math

import numpy as np
import pytest

from oracle.basis import gauss, gll, lagrange, lagrange_deriv, mass_1d, stiff_1d

# Gauss-Lobatto-Legendre nodes and weights in closed form (textbook values)
GLL_CLOSED = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
        [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("p", sorted(GLL_CLOSED))
def test_gll_closed_form(p):
    x, w = gll(p)
    xe, we = GLL_CLOSED[p]
    assert np.allclose(x, xe, atol=1e-15, rtol=0)
    assert np.allclose(w, we, atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_gll_exactness(p):
    # the (p+1)-point Lobatto rule integrates degree <= 2p-1 exactly
    x, w = gll(p)
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("q", [1, 2, 3, 4, 7])
def test_gauss_exactness(q):
    x, w = gauss(q)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_lagrange_cardinal_and_derivative(p):
    r, _ = gll(p)
    assert np.allclose(lagrange(r, r), np.eye(p + 1), atol=1e-14)
    # derivative of an interpolated polynomial of degree p is exact
    xs = np.linspace(-1, 1, 11)
    coef = np.arange(1, p + 2, dtype=float)
    poly = np.polynomial.Polynomial(coef)
    vals = lagrange_deriv(r, xs) @ poly(r)
    assert np.allclose(vals, poly.deriv()(xs), atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_integration_by_parts_identity(p):
    # int l_a' l_b + int l_a l_b' = l_a(1) l_b(1) - l_a(-1) l_b(-1)
    S = stiff_1d(p)
    E = np.zeros((p + 1, p + 1))
    E[p, p], E[0, 0] = 1.0, -1.0
    assert np.abs(S + S.T - E).max() < 1e-13
    assert abs(mass_1d(p).sum() - 2.0) < 1e-14
