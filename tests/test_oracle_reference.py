"""Pins for the oracle's reference-element operators (Sections 2.3, 2.4, 3, 4.3, 5.1)."""
import itertools
import json
import os
from functools import lru_cache

import numpy as np
import pytest
import sympy

from oracle.reference import RefElement, collapse
from oracle.pkd import vandermonde, pkd_eval, modal_indices

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CASES = [(2, q) for q in (1, 2, 3, 4, 6, 8)] + [(3, q) for q in (1, 2, 3, 4)]


@lru_cache(maxsize=None)
def ref(dim, q):
    return RefElement(dim, q)


@lru_cache(maxsize=None)
def simplex_monomial_integral(dim, powers):
    """Exact integral of xi^powers over the reference simplex (symbolic, iterated limits)."""
    x = sympy.symbols("x1:4")
    f = sympy.Integer(1)
    for k, pw in enumerate(powers):
        f *= x[k] ** pw
    if dim == 2:
        val = sympy.integrate(f, (x[0], -1, -x[1]), (x[1], -1, 1))
    else:
        val = sympy.integrate(f, (x[0], -1, -1 - x[1] - x[2]), (x[1], -1, -x[2]), (x[2], -1, 1))
    return float(val)


def monomials(dim, deg):
    return [a for a in itertools.product(range(deg + 1), repeat=dim) if sum(a) <= deg]


@pytest.mark.parametrize("dim,q", CASES)
def test_sbp_property(dim, q):
    """Q^(l) + Q^(l)T = E^(l) = sum_zeta nhat_l R^T B R (Definition 2, Eq. (e_decomp))."""
    r = ref(dim, q)
    for l in range(dim):
        assert np.abs(r.Q[l] + r.Q[l].T - r.E[l]).max() < 1e-13 * max(1, np.abs(r.Q[l]).max())
        assert np.abs(r.S[l] + r.S[l].T).max() == 0.0


@pytest.mark.parametrize("dim,q", CASES)
def test_derivative_exactness(dim, q):
    """D^(l) differentiates every polynomial of total degree <= q exactly (Eq. (accuracy))."""
    r = ref(dim, q)
    for a in monomials(dim, q):
        v = np.prod(r.xi ** np.array(a), axis=1)
        for l in range(dim):
            if a[l] == 0:
                dv = np.zeros(r.Nq)
            else:
                b = list(a); b[l] -= 1
                dv = a[l] * np.prod(r.xi ** np.array(b), axis=1)
            assert np.abs(r.D[l] @ v - dv).max() < 1e-11


@pytest.mark.parametrize("dim,q", CASES)
def test_extrapolation_exactness(dim, q):
    """R^(zeta) reproduces every polynomial of degree <= q at the facet nodes (Eq. (extrap_acc))."""
    r = ref(dim, q)
    for a in monomials(dim, q):
        v = np.prod(r.xi ** np.array(a), axis=1)
        for z in range(r.Nf):
            assert np.abs(r.R[z] @ v - np.prod(r.xif[z] ** np.array(a), axis=1)).max() < 1e-12


@pytest.mark.parametrize("dim,q", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_volume_quadrature_degree_2q(dim, q):
    """The tensor-product rule integrates P_2q exactly (Eq. (sbp_quadrature), degree tau >= 2q-1)."""
    r = ref(dim, q)
    for a in monomials(dim, 2 * q):
        exact = simplex_monomial_integral(dim, a)
        assert abs(np.sum(r.w * np.prod(r.xi ** np.array(a), axis=1)) - exact) < 1e-13


@pytest.mark.parametrize("dim,q", CASES)
def test_facet_measures_and_nodes(dim, q):
    """Facet weights sum to the facet measure; facet nodes lie on the facet (Eq. (tri_facets), Eq. (tet_facets))."""
    r = ref(dim, q)
    if dim == 2:
        meas = [2.0, 2.0 * np.sqrt(2.0), 2.0]
        on = [lambda x: x[:, 1] + 1, lambda x: x[:, 0] + x[:, 1], lambda x: x[:, 0] + 1]
    else:
        meas = [2.0, 2.0 * np.sqrt(3.0), 2.0, 2.0]
        on = [lambda x: x[:, 1] + 1, lambda x: x.sum(1) + 1, lambda x: x[:, 0] + 1, lambda x: x[:, 2] + 1]
    for z in range(r.Nf):
        assert abs(r.wf[z].sum() - meas[z]) < 1e-13
        assert np.abs(on[z](r.xif[z])).max() < 1e-14
        assert np.abs(np.linalg.norm(r.nhat[z]) - 1) < 1e-15
    assert abs(r.w.sum() - (2.0 if dim == 2 else 4.0 / 3.0)) < 1e-14


@pytest.mark.parametrize("dim,q", [(2, 1), (2, 3), (3, 1), (3, 2)])
def test_facet_quadrature_exactness(dim, q):
    """Facet rules integrate degree-2q polynomials exactly over each facet (checked by the
    divergence theorem: sum_zeta nhat_l int_facet f = int_volume df/dxi_l)."""
    r = ref(dim, q)
    for a in monomials(dim, 2 * q + 1):
        for l in range(dim):
            if a[l] == 0:
                continue
            b = list(a); b[l] -= 1
            vol = a[l] * simplex_monomial_integral(dim, tuple(b))
            surf = sum(r.nhat[z][l] * np.sum(r.wf[z] * np.prod(r.xif[z] ** np.array(a), axis=1))
                       for z in range(r.Nf))
            assert abs(surf - vol) < 1e-12


def _counts(r):
    vol = sum(np.count_nonzero(S) // 2 for S in r.S)
    fac = sum(np.count_nonzero(R.T @ B) for R, B in zip(r.R, r.B))
    return vol, fac


@pytest.mark.parametrize("dim,q", [(2, q) for q in (2, 3, 4, 5, 6, 10)] + [(3, q) for q in (2, 3, 4)])
def test_flux_counts_match_paper_formula(dim, q):
    """Eq. (num_fluxes) with the tensor-product sparsity: golden counts (Section 5.1)."""
    gold = json.load(open(os.path.join(GOLD, "flux_counts.json")))
    r = ref(dim, q)
    vol, fac = _counts(r)
    key = "triangle" if dim == 2 else "tetrahedron"
    assert vol + fac == gold[key][str(q)]
    if dim == 2:
        assert vol == q * (q + 1) ** 2 // 2 + q * (q + 1) ** 2
        assert fac == 3 * (q + 1) ** 2
    else:
        assert vol == 3 * q * (q + 1) ** 3
        assert fac == 3 * (q + 1) ** 3 + (q + 1) ** 4


def test_printed_reduction_factors_q2():
    """The printed q = 2 reduction factors (1.56 triangles, 1.88 tetrahedra) follow from our counts."""
    gold = json.load(open(os.path.join(GOLD, "flux_counts.json")))["printed_reduction_q2"]
    for dim, key in ((2, "triangle"), (3, "tetrahedron")):
        g = gold[key]
        multi = dim * g["N"] * (g["N"] - 1) // 2 + g["n_facets"] * g["N"] * g["Nf_nodes"]
        vol, fac = _counts(ref(dim, 2))
        assert round(multi / (vol + fac), 2) == g["printed"]


@pytest.mark.parametrize("dim,p", [(2, p) for p in (1, 2, 4, 7, 10)] + [(3, p) for p in (1, 2, 4, 6)])
def test_pkd_orthonormal(dim, p):
    """M = V^T W V = I for the normalized PKD basis (Section 4.3)."""
    r = ref(dim, p) if (dim, p) in CASES else RefElement(dim, p)
    V = vandermonde(r, p)
    assert V.shape == (r.Nq, len(modal_indices(dim, p)))
    assert np.abs(V.T @ r.W @ V - np.eye(V.shape[1])).max() < 1e-12


@pytest.mark.parametrize("dim,p", [(2, 3), (2, 5), (3, 2), (3, 3)])
def test_pkd_spans_total_degree_space(dim, p):
    """Every monomial of degree <= p is reproduced by the PKD expansion (least squares is exact)."""
    r = RefElement(dim, p)
    V = vandermonde(r, p)
    for a in monomials(dim, p):
        v = np.prod(r.xi ** np.array(a), axis=1)
        c = V.T @ r.W @ v
        assert np.abs(V @ c - v).max() < 1e-12
    # the constant mode is 1/sqrt(|Omega|)
    phi0 = pkd_eval(dim, p, r.eta[:3])[:, 0]
    assert np.allclose(phi0, 1 / np.sqrt(2.0 if dim == 2 else 4.0 / 3.0))


def test_collapse_maps_vertices():
    """chi maps the square/cube onto the reference simplex; the tetrahedron map, read with
    (1 - eta_3) as the third factor of xi_1 where the print repeats (1 - eta_2), sends cube
    vertices to simplex vertices and the Jacobian determinant matches the weights."""
    tri = collapse(np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], float))
    assert np.allclose(tri, [[-1, -1], [1, -1], [-1, 1], [-1, 1]])
    cube = np.array(list(itertools.product([-1.0, 1.0], repeat=3)))
    img = collapse(cube)
    assert np.all(img.sum(1) <= -1 + 1e-14)
    verts = {tuple(v) for v in np.round(img, 12)}
    assert verts == {(-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)}


def _lg_sbp_1d(q):
    """The 1D Legendre-Gauss SBP operator Q1 = diag(w) D1 (Section 2.4) built from numpy's
    Legendre routines alone: D1 = V' V^{-1} with the Legendre Vandermonde V on the nodes."""
    leg = np.polynomial.legendre
    x, w = leg.leggauss(q + 1)
    V = leg.legvander(x, q)
    dV = np.stack([leg.legval(x, leg.legder(np.eye(q + 1)[k])) for k in range(q + 1)], axis=1)
    D1 = dV @ np.linalg.inv(V)
    tL = leg.legvander(np.array([-1.0]), q)[0] @ np.linalg.inv(V)   # extrapolation to -1
    tR = leg.legvander(np.array([1.0]), q)[0] @ np.linalg.inv(V)    # extrapolation to +1
    return x, w, np.diag(w) @ D1, tL, tR


def test_q1_eta1_line_operator_by_hand():
    """q = 1 by hand: LG nodes -+1/sqrt(3), weights 1, linear Lagrange derivatives -+sqrt(3)/2,
    so the 1D operator is (sqrt(3)/2)[[-1, 1], [-1, 1]] and Q1 + Q1^T = diag(-sqrt(3), sqrt(3)).
    On the triangle (Eq. (tri_quadrature), Eq. (d1_2d)) the factor (1 - eta_2)/2 of the weight
    cancels 2/(1 - eta_2) of D^(1), so each eta_1 line of Q^(1) = W D^(1) is w_2 Q1 = Q1."""
    s = np.sqrt(3.0) / 2
    Q1 = s * np.array([[-1.0, 1.0], [-1.0, 1.0]])
    assert np.allclose(Q1 + Q1.T, np.diag([-np.sqrt(3.0), np.sqrt(3.0)]), atol=1e-15)
    r = ref(2, 1)
    for a2 in range(2):
        line = [a1 * 2 + a2 for a1 in range(2)]   # alpha_1 slowest
        assert np.abs(r.Q[0][np.ix_(line, line)] - Q1).max() < 1e-14
    off = [(i, j) for i in range(4) for j in range(4) if (i % 2) != (j % 2)]
    assert all(r.Q[0][i, j] == 0.0 for i, j in off)


@pytest.mark.parametrize("dim,q", [(2, q) for q in (2, 3, 5, 8)] + [(3, q) for q in (2, 3, 4)])
def test_eta1_lines_are_scaled_1d_lg_sbp(dim, q):
    """The eta_1 lines of Q^(1) are scaled copies of the 1D LG SBP operator: on the triangle the
    weight factor (1 - eta_2)/2 cancels 2/(1 - eta_2) of Eq. (d1_2d), leaving w_2(alpha_2) Q1;
    on the tetrahedron (1 - eta_2)(1 - eta_3)/8 against 4/((1 - eta_2)(1 - eta_3)) of Eq. (d_3d)
    leaves w_2(alpha_2) w_3(alpha_3)/2 Q1, with w_3 the Gauss-Jacobi(1,0) weights.  Q1 itself
    satisfies Q1 + Q1^T = tR tR^T - tL tL^T (the 1D SBP property)."""
    from scipy.special import roots_jacobi
    x, w, Q1, tL, tR = _lg_sbp_1d(q)
    assert np.abs(Q1 + Q1.T - (np.outer(tR, tR) - np.outer(tL, tL))).max() < 1e-12
    r = ref(dim, q) if (dim, q) in CASES else RefElement(dim, q)
    n = q + 1
    Q = r.Q[0]
    scale = np.abs(Q1).max()
    if dim == 2:
        lines = [((a2,), w[a2]) for a2 in range(n)]
    else:
        _, w3 = roots_jacobi(n, 1.0, 0.0)
        lines = [((a2, a3), w[a2] * w3[a3] / 2) for a2 in range(n) for a3 in range(n)]
    seen = np.zeros_like(Q, dtype=bool)
    for rest, c in lines:
        idx = [int(np.ravel_multi_index((a1,) + rest, (n,) * dim)) for a1 in range(n)]
        assert np.abs(Q[np.ix_(idx, idx)] - c * Q1).max() < 1e-12 * scale
        seen[np.ix_(idx, idx)] = True
    assert np.all(Q[~seen] == 0.0)
