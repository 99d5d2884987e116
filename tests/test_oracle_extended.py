"""Pins for the oracle in extended precision (np.longdouble): the route that gives the
exact answer against which the FP64 implementations (the oracle and the CUDA library) are
measured.  Each check is one that FP64 arithmetic cannot pass, so it shows both that the
formulas are right and that the extra precision is really carried through."""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import esd_inputs as I
from oracle import euler, extended
from oracle.jacobi import gauss_jacobi
from oracle.pkd import vandermonde
from oracle.reference import RefElement
from oracle.residual import Discretization

X = np.longdouble
EPS = np.finfo(X).eps
FP64_EPS = np.finfo(np.float64).eps
pytestmark = pytest.mark.skipif(EPS >= FP64_EPS / 100, reason="no extended long double on this platform")


def jacobi_moment(k, a, b):
    """int_{-1}^{1} x^k (1-x)^a (1+x)^b dx, exactly: with x = 2t - 1 it is
    2^(a+b+1) sum_j C(k,j) 2^j (-1)^(k-j) B(j+b+1, a+1), B of integers = a rational."""
    beta = lambda m, n: Fraction(factorial(m - 1) * factorial(n - 1), factorial(m + n - 1))
    s = sum(comb(k, j) * 2 ** j * (-1) ** (k - j) * beta(j + b + 1, a + 1) for j in range(k + 1))
    return 2 ** (a + b + 1) * s


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (5, 0)])
@pytest.mark.parametrize("q", [1, 4, 10])
def test_gauss_jacobi_exact_in_long_double(q, a, b):
    """Section 2.5: the (q+1)-node rule integrates x^k (k <= 2q+1) exactly; in long double
    to a few long-double ulps, which the FP64 rule misses by orders of magnitude."""
    x, w = gauss_jacobi(q, a, b, X)
    x64, w64 = gauss_jacobi(q, a, b)
    assert x.dtype == X and w.dtype == X
    worst, worst64 = 0.0, 0.0
    for k in range(2 * q + 2):
        m = jacobi_moment(k, a, b)
        exact = X(m.numerator) / X(m.denominator)
        scale = X(np.sum(np.abs(w) * np.abs(x) ** k))
        worst = max(worst, abs(np.sum(w * x ** k) - exact) / scale)
        worst64 = max(worst64, abs(np.sum(w64.astype(X) * x64.astype(X) ** k) - exact) / scale)
    assert worst < 64 * EPS, worst
    assert worst64 > 64 * EPS          # the bound discriminates FP64 from long double


@pytest.mark.parametrize("dim,p", [(2, 3), (2, 8), (3, 2), (3, 5)])
def test_pkd_orthonormal_in_long_double(dim, p):
    """Section 4.3: V^T W V = I (the PKD basis is orthonormal under the volume rule)."""
    ref = RefElement(dim, p, X)
    V = vandermonde(ref, p)
    assert V.dtype == X
    G = V.T @ (ref.w[:, None] * V)
    assert np.abs(G - np.eye(G.shape[0], dtype=X)).max() < 256 * EPS


@pytest.mark.parametrize("dim,q", [(2, 3), (3, 2)])
def test_sbp_property_in_long_double(dim, q):
    """Definition 2 / Eq. (e_decomp): Q^(l) + Q^(l)T = sum_zeta nhat_l R^T B R, and D exact on
    monomials of degree <= q, in long double."""
    ref = RefElement(dim, q, X)
    for l in range(dim):
        Q, E = ref.Q[l], ref.E[l]
        assert np.abs(Q + Q.T - E).max() < 256 * EPS * np.abs(Q).max()
    x = ref.xi
    for l in range(dim):
        for powers in [(1, 0, 0), (0, 1, 0), (q, 0, 0), (0, q - 1, 1), (1, 1, q - 2)]:
            powers = powers[:dim]
            if sum(powers) > q or min(powers) < 0:
                continue
            f = np.prod([x[:, k] ** powers[k] for k in range(dim)], axis=0)
            df = powers[l] * np.prod([x[:, k] ** (powers[k] - (k == l)) if powers[k] - (k == l) >= 0 else 0 * x[:, k]
                                      for k in range(dim)], axis=0)
            assert np.abs(ref.D[l] @ f - df).max() < 1024 * EPS * max(1, np.abs(df).max())


def test_log_mean_in_long_double():
    """Section 7.2: {{a}}_ln = (b - a)/ln(b/a) in both branches, against 40-digit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    a = rng.uniform(0.1, 10, 400)
    rel = np.concatenate([rng.uniform(-1e-3, 1e-3, 200), rng.uniform(-0.9, 0.9, 200)])
    b = a * (1 + rel)
    aX, bX = a.astype(X), b.astype(X)
    lm = euler.log_mean(aX, bX)
    ilm = euler.inv_log_mean(aX, bX)
    for i in range(len(a)):
        A, B = mpmath.mpf(float(a[i])), mpmath.mpf(float(b[i]))
        exact = (B - A) / mpmath.log(B / A) if A != B else A
        tol = 16 * EPS * (1 + 1 / abs(np.log(b[i] / a[i])))
        assert abs(float((mpmath.mpf(str(lm[i])) - exact) / exact)) < tol
        assert abs(float((mpmath.mpf(str(ilm[i])) - 1 / exact) * exact)) < tol


def test_entropy_variables_round_trip_in_long_double():
    """Section 7.1: U(W(u)) = u to long-double rounding."""
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.2, 3, 200)
    v = rng.uniform(-2, 2, (200, 3))
    p = rng.uniform(0.2, 80, 200)
    u = euler.conservative(rho.astype(X), v.astype(X), p.astype(X))
    back = euler.cons_from_entropy(euler.entropy_vars(u))
    assert back.dtype == X
    assert np.abs(back - u).max() < 1e3 * EPS * np.abs(u).max()


def small(dim, M, p, warp=True, flux="LF", state=None):
    L = 2 * np.pi
    mesh, Xn = I.config_mesh(dim, M, L, p, warp)
    D = Discretization(dim, p, Xn, mesh.nbr_elem, mesh.nbr_face, flux=flux)
    f = I.config_state_fn(dim, L, state or ("vortex" if dim == 2 else "tgv"))
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, f(D.geo.x_vol)) + I.seeded_normal(5, (D.E, dim + 2, D.Np), 1e-3)
    return mesh, Xn, D, um


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2)])
def test_free_stream_in_long_double(dim, p):
    """Theorem 3: a uniform state has d u~/dt = 0 on curved periodic meshes -- in long
    double to long-double rounding (FP64 reaches only ~1e-15)."""
    mesh, Xn, D, _ = small(dim, 3, p)
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7, 0.2][:dim]), np.array(2.1))
    um = np.zeros((D.E, D.Nc, D.Np))
    um[:, :, 0] = ubar / D.V[0, 0]       # only the constant mode: exactly uniform at every node
    el = np.array([0, 7, 11])
    r = extended.rhs(D, Xn, um, el)
    assert r.dtype == X
    assert np.abs(r).max() < 4096 * EPS * np.abs(ubar).max()


@pytest.mark.parametrize("flux", ["EC", "LF"])
def test_conservation_and_entropy_in_long_double(flux):
    """Theorems 2 and 4 on the whole mesh in long double: sum 1^T W J V d u~/dt = 0 and, with
    the entropy-conservative interface flux, sum w^T W J V d u~/dt = 0 (with LF: < 0), each
    to long-double rounding of its scale."""
    mesh, Xn, D, um = small(2, 3, 2, True, flux)
    Dx = Discretization(2, 2, Xn.astype(X), mesh.nbr_elem, mesh.nbr_face, flux=flux, dtype=X)
    umx = um.astype(X)
    dudt = Dx.rhs(umx, "sparse")
    cons = Dx.conservation_rate(dudt)
    y = np.einsum("ij,ecj->eic", Dx.V, dudt)
    scale = np.einsum("i,ei,eic->c", Dx.ref.w, Dx.geo.J_vol, np.abs(y))
    assert np.all(np.abs(cons) < 1024 * EPS * scale)
    ent, ent_scale = Dx.entropy_rate(umx, dudt)
    if flux == "EC":
        assert abs(ent) < 1024 * EPS * ent_scale
    else:
        assert ent < -1e-6 * ent_scale


@pytest.mark.parametrize("dim,p,state", [(2, 3, "vortex"), (3, 2, "density_wave"), (3, 3, "tgv")])
def test_extended_route_is_the_fp64_route(dim, p, state):
    """The long-double evaluation on a sub-mesh equals (i) the long-double evaluation of
    the whole mesh, bit for bit, and (ii) the FP64 oracle within FP64 rounding of the term
    scale (the sums of |terms|)."""
    mesh, Xn, D, um = small(dim, 3, p, state=state)
    el = np.array([2, 9, 13])
    rx, scale = extended.rhs_and_scale(D, Xn, um, el)
    Dx = Discretization(dim, p, Xn.astype(X), mesh.nbr_elem, mesh.nbr_face, dtype=X)
    full = Dx.rhs(um.astype(X), "sparse", elems=el)
    assert np.array_equal(rx, full)
    r64 = D.rhs(um, "sparse", elems=el)
    assert np.all(scale >= np.abs(rx))
    err = np.abs(r64 - rx) / scale
    assert err.max() < 1e-13, err.max()
    # the FP64 oracle is NOT exact: its error is far above long-double rounding
    assert np.abs(r64 - rx).max() > 1e3 * EPS * np.abs(rx).max()


def test_extended_projection_matches_fp64():
    """Eq. (entropy_expansion) in long double agrees with the FP64 projection to FP64 rounding."""
    mesh, Xn, D, um = small(3, 3, 3)
    el = np.array([1, 4])
    wx = extended.project_entropy(D, Xn, um, el)
    w64 = D.project_entropy(um, el)
    assert wx.dtype == X
    assert np.abs(w64 - wx).max() < 1e-13 * np.abs(wx).max()


def test_sub_discretization_matches_whole_mesh():
    """A sub-mesh built from the mesh arrays alone (facets matched inside it) gives the same
    d u~/dt for its central elements as the whole mesh, in FP64 bit for bit."""
    mesh, Xn, D, um = small(3, 3, 2, state="density_wave")
    el = np.array([5, 40, 161])
    Ds, need, local = extended.sub_discretization(3, 2, Xn, mesh.nbr_elem, mesh.nbr_face, el, dtype=np.float64)
    got = Ds.rhs(um[need], "sparse", elems=local)
    assert np.array_equal(got, D.rhs(um, "sparse", elems=el))
    assert np.array_equal(Ds.geo.perm[local], D.geo.perm[el])
