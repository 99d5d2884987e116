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
