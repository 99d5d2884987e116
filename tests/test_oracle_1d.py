"""Pins for the oracle's Section 2.5 building blocks (Jacobi polynomials, Gauss rules, Lagrange)."""
import json
import os
from fractions import Fraction
from math import gamma as G, sqrt

import numpy as np
import pytest
import scipy.special as sp

from oracle.jacobi import jacobi_p, gauss_jacobi, lagrange, lagrange_deriv

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _norm2(n, a, b):
    """Squared L2 norm of scipy's (unnormalized) Jacobi polynomial under (1-x)^a(1+x)^b."""
    return 2 ** (a + b + 1) / (2 * n + a + b + 1) * G(n + a + 1) * G(n + b + 1) / (G(n + a + b + 1) * G(n + 1))


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (3, 0), (5, 0), (8, 0)])
def test_jacobi_matches_library(a, b):
    x = np.linspace(-1, 1, 37)
    P = jacobi_p(9, a, b, x)
    for n in range(10):
        ref = sp.eval_jacobi(n, a, b, x) / sqrt(_norm2(n, a, b))
        assert np.allclose(P[n], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0)])
@pytest.mark.parametrize("q", range(0, 12))
def test_gauss_jacobi_matches_library(q, a, b):
    x, w = gauss_jacobi(q, a, b)
    xr, wr = sp.roots_jacobi(q + 1, a, b)
    assert np.allclose(np.sort(x), np.sort(xr), atol=1e-14)
    assert np.allclose(w[np.argsort(x)], wr[np.argsort(xr)], rtol=1e-12)


def _moment(k, a, b):
    """Exact int_{-1}^{1} x^k (1-x)^a (1+x)^b dx for integer a, b (binomial expansion, rationals)."""
    tot = Fraction(0)
    from math import comb
    # (1-x)^a (1+x)^b = sum_{i,j} C(a,i)(-1)^i C(b,j) x^(i+j)
    for i in range(a + 1):
        for j in range(b + 1):
            e = k + i + j
            if e % 2 == 0:
                tot += comb(a, i) * (-1) ** i * comb(b, j) * Fraction(2, e + 1)
    return float(tot)


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0)])
@pytest.mark.parametrize("q", [0, 1, 2, 4, 7, 10])
def test_gauss_exactness_degree_2q_plus_1(q, a, b):
    x, w = gauss_jacobi(q, a, b)
    for k in range(2 * q + 2):
        assert abs(np.sum(w * x ** k) - _moment(k, a, b)) < 1e-13 * max(1.0, abs(_moment(k, a, b)))
    # and not exact one degree higher (it is a Gauss rule, not a higher one)
    k = 2 * q + 2
    assert abs(np.sum(w * x ** k) - _moment(k, a, b)) > 1e-10


def test_gauss_golden_closed_forms():
    gold = json.load(open(os.path.join(GOLD, "gauss_rules.json")))
    env = {"sqrt": np.sqrt}
    for q, rec in gold["legendre"].items():
        x, w = gauss_jacobi(int(q), 0, 0)
        o = np.argsort(x)
        assert np.allclose(x[o], [eval(s, env) for s in rec["nodes"]], atol=1e-15)
        assert np.allclose(w[o], [eval(s, env) for s in rec["weights"]], atol=1e-15)
    for q in ("0", "1"):
        rec = gold["jacobi_1_0"][q]
        x, w = gauss_jacobi(int(q), 1, 0)
        assert np.allclose(np.sort(x), [eval(s, env) for s in rec["nodes"]], atol=1e-15)
        if "weights" in rec:
            assert np.allclose(w, [eval(s, env) for s in rec["weights"]], atol=1e-15)


@pytest.mark.parametrize("q", [1, 3, 6, 10])
def test_lagrange_cardinal_and_derivative_exact(q):
    x, _ = gauss_jacobi(q, 0, 0)
    assert np.allclose(lagrange(x, x), np.eye(q + 1), atol=1e-13)
    t = np.linspace(-1, 1, 13)
    rng = np.random.default_rng(0)
    c = rng.normal(size=q + 1)
    poly = np.polynomial.Polynomial(c)
    # derivative of the interpolant of a degree-q polynomial equals its derivative
    d = lagrange_deriv(x, t).T @ poly(x)
    assert np.allclose(d, poly.deriv()(t), rtol=1e-10, atol=1e-10)
    v = lagrange(x, t).T @ poly(x)
    assert np.allclose(v, poly(t), rtol=1e-11, atol=1e-11)
