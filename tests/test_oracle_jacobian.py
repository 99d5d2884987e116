"""Pins for the oracle's complex-step Jacobian (the VJP reference): agreement with central
finite differences of the real oracle, linearity, and the element-local structure."""
from functools import lru_cache

import numpy as np
import pytest

import esd_inputs as I
from oracle.residual import Discretization
from oracle.jacobian import jvp, local_vjp, rk4_jvp
from oracle.timestep import rk4_step


@lru_cache(maxsize=None)
def disc(dim, p, state, flux="LF"):
    L = 2 * np.pi
    mesh, X = I.config_mesh(dim, 3, L, p, True)
    D = Discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux=flux)
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, I.config_state_fn(dim, L, state)(D.geo.x_vol))
    return D, um + I.seeded_normal(4, um.shape, 1e-3)


@pytest.mark.parametrize("dim,p,state", [(2, 2, "vortex"), (2, 3, "vortex"), (3, 2, "density_wave")])
@pytest.mark.parametrize("flux", ["LF", "EC"])
def test_complex_step_matches_central_differences(dim, p, state, flux):
    D, um = disc(dim, p, state, flux)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(um.shape)
    el = np.arange(min(D.E, 10))
    jv = jvp(D, um, v, elems=el)
    h = 1e-6
    fd = (D.rhs(um + h * v, "sparse", elems=el) - D.rhs(um - h * v, "sparse", elems=el)) / (2 * h)
    assert np.abs(jv - fd).max() < 1e-6 * np.abs(jv).max()


def test_jvp_is_linear_and_local():
    D, um = disc(2, 2, "vortex")
    rng = np.random.default_rng(1)
    v1, v2 = rng.standard_normal(um.shape), rng.standard_normal(um.shape)
    a = jvp(D, um, 2.0 * v1 - 3.0 * v2)
    b = 2.0 * jvp(D, um, v1) - 3.0 * jvp(D, um, v2)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    e = 4
    v = np.zeros(um.shape)
    v[e] = rng.standard_normal(um.shape[1:])
    col = jvp(D, um, v)
    far = np.setdiff1d(np.arange(D.E), np.concatenate([[e], D.geo.nbr_elem[e]]))
    assert np.abs(col[far]).max() == 0.0


def test_local_vjp_is_transpose():
    D, um = disc(2, 2, "vortex")
    rng = np.random.default_rng(2)
    cot = rng.standard_normal(um.shape)
    e = 3
    g = local_vjp(D, um, cot, e)
    v = np.zeros(um.shape)
    v[e] = rng.standard_normal(um.shape[1:])
    assert abs(np.sum(g * v[e]) - np.sum(cot * jvp(D, um, v))) < 1e-11 * np.abs(g).sum()


def test_rk4_jvp_against_differences():
    D, um = disc(2, 2, "vortex")
    rng = np.random.default_rng(3)
    v = rng.standard_normal(um.shape)
    dt = 1e-3
    jv = rk4_jvp(D, um, v, dt)
    h = 1e-6
    f = lambda x: rk4_step(lambda y: D.rhs(y, "sparse"), x, dt)
    fd = (f(um + h * v) - f(um - h * v)) / (2 * h)
    assert np.abs(jv - fd).max() < 1e-6 * np.abs(jv).max()


@pytest.mark.parametrize("dim,p,state", [(2, 2, "vortex"), (3, 2, "density_wave")])
def test_batched_local_vjp_equals_column_by_column(dim, p, state):
    """local_vjp_batched (all columns at once on copies of the neighbourhood) equals the
    column-by-column local_vjp to rounding, also for an element on a periodic face."""
    from oracle.jacobian import local_vjp_batched
    D, um = disc(dim, p, state)
    rng = np.random.default_rng(5)
    cot = rng.standard_normal(um.shape)
    for e in (0, D.E - 1):
        a = local_vjp(D, um, cot, e)
        b = local_vjp_batched(D, um, cot, e)
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


def test_batched_local_vjp_in_long_double():
    """In long double (complex long double steps) on a sub-mesh, the batched local VJP agrees
    with FP64 to FP64 rounding and is itself a transpose to long-double rounding."""
    from oracle import extended
    from oracle.jacobian import local_vjp_batched
    X = np.longdouble
    if np.finfo(X).eps >= np.finfo(float).eps / 100:
        pytest.skip("no extended long double")
    L = 2 * np.pi
    mesh, Xn = I.config_mesh(2, 3, L, 2, True)
    D, um = disc(2, 2, "vortex")
    rng = np.random.default_rng(6)
    cot = rng.standard_normal(um.shape)
    e = 7
    nb = np.unique(np.concatenate([[e], D.geo.nbr_elem[e]]))
    ring = np.unique(np.concatenate([nb, D.geo.nbr_elem[nb].ravel()]))
    Dx, need, local = extended.discretization(D, Xn, ring)
    ie = int(np.searchsorted(need, e))
    gx = local_vjp_batched(Dx, um[need], cot[need], ie)
    g64 = local_vjp_batched(D, um, cot, e)
    assert gx.dtype == X
    assert np.abs(gx - g64).max() < 1e-12 * np.abs(gx).max()
    v = rng.standard_normal(um.shape[1:])
    U = um[need].astype(np.clongdouble)
    U[ie] += 1j * 1e-30 * v
    inb = np.searchsorted(need, nb)
    jv = np.imag(Dx.rhs(U, "sparse", elems=inb)) / 1e-30
    lhs, rhs = np.sum(gx * v), np.sum(cot[nb].astype(X) * jv)
    assert abs(lhs - rhs) < 1e3 * np.finfo(X).eps * np.sum(np.abs(gx * v))
