"""Pins for the oracle's conservative and skew-symmetric forms (Section 4.4, Eq. (rhs_cons),
Eq. (rhs_skew)): they coincide on affine meshes; the skew-symmetric form preserves a
uniform state and conserves on curved meshes, and for linear advection it conserves the
discrete energy u^T r (central flux) or dissipates it (upwind) on curved meshes, which
the conservative form does not."""
from functools import lru_cache

import numpy as np
import pytest

import esd_inputs as I
from oracle import euler, skew
from oracle.residual import Discretization


@lru_cache(maxsize=None)
def disc(dim, M, p, warp):
    L = 2 * np.pi
    mesh, X = I.config_mesh(dim, M, L, p, warp)
    return Discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face)


def euler_state(D, seed):
    f = I.config_state_fn(D.dim, 2 * np.pi, "vortex" if D.dim == 2 else "tgv")
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, f(D.geo.x_vol))
    return um + I.seeded_normal(seed, um.shape, 1e-3)


CASES = [(2, 3, 2), (2, 3, 4), (3, 3, 2)]


@pytest.mark.parametrize("dim,M,p", CASES)
def test_forms_coincide_on_affine_meshes(dim, M, p):
    """With constant metrics G^(l,m) and J^zeta n = G^T nhat, the SBP property turns
    Eq. (rhs_skew) into Eq. (rhs_cons) exactly; on curved meshes whose metric terms are
    not affine functions of xi (sine-warped, p >= 3 triangles, p >= 2 tetrahedra with the
    curl-form metrics) they differ."""
    model = skew.EulerModel(dim)
    D = disc(dim, M, p, False)
    um = euler_state(D, 3)
    el = np.arange(min(D.E, 12))
    a = skew.nodal_residual(D, um, model, "skew", el)
    b = skew.nodal_residual(D, um, model, "cons", el)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()
    if dim == 2 and p < 3:
        return
    Dc = disc(dim, M, p, True)
    umc = euler_state(Dc, 3)
    a = skew.nodal_residual(Dc, umc, model, "skew", el)
    b = skew.nodal_residual(Dc, umc, model, "cons", el)
    assert np.abs(a - b).max() > 1e-8 * np.abs(b).max()


@pytest.mark.parametrize("dim,M,p", CASES)
def test_skew_free_stream_on_curved_meshes(dim, M, p):
    """A uniform state gives r = 0: Q 1 = 0, the discrete metric identities, and R exact
    on the metric terms cancel the volume against the facet terms."""
    D = disc(dim, M, p, True)
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7, 0.2][:dim]), np.array(2.1))
    un = np.broadcast_to(ubar, (D.E, D.ref.Nq, D.Nc))
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, un)
    r = skew.nodal_residual(D, um, skew.EulerModel(dim), "skew", np.arange(min(D.E, 20)))
    assert np.abs(r).max() < 1e-12 * np.abs(ubar).max()


@pytest.mark.parametrize("dim,M,p", CASES)
def test_skew_conservation_on_curved_meshes(dim, M, p):
    """sum_kappa 1^T r = -sum_kappa sum_zeta 1^T B J^zeta f* = 0 on a periodic mesh, and the
    same for sum_kappa 1^T W J V d u~/dt through the weight-adjusted inverse."""
    D = disc(dim, M, p, True)
    model = skew.EulerModel(dim)
    um = euler_state(D, 5)
    r = skew.nodal_residual(D, um, model, "skew")
    scale = np.abs(r).sum(axis=(0, 1))
    assert np.all(np.abs(r.sum(axis=(0, 1))) < 1e-13 * scale)
    dudt = skew.rhs(D, um, model, "skew")
    rate = D.conservation_rate(dudt)
    y = np.einsum("ij,ecj->eic", D.V, dudt)
    scale = np.einsum("i,ei,eic->c", D.ref.w, D.geo.J_vol, np.abs(y))
    assert np.all(np.abs(rate) < 1e-13 * scale)


@pytest.mark.parametrize("dim,M,p", CASES + [(3, 3, 3)])
def test_skew_energy_for_linear_advection_on_curved_meshes(dim, M, p):
    """f_m = a_m u: the skew-symmetric volume terms cancel in u^T r for any metric terms, so
    with the central interface flux sum_kappa u^T r = 0 (d/dt of the weight-adjusted energy
    u~^T M~ u~ / 2) and with upwinding it is negative.  The conservative form has no such
    identity once the metric terms are of higher degree (checked at p >= 3 here)."""
    D = disc(dim, M, p, True)
    a = np.array([1.0, 0.5, -0.3][:dim])
    um = I.seeded_normal(9, (D.E, 1, D.Np), 1.0)
    u, _ = skew.nodal_states(D, um)

    def energy_rate(model, form):
        r = skew.nodal_residual(D, um, model, form)
        return float(np.sum(u * r)), float(np.sum(np.abs(u * r)))

    ent, scale = energy_rate(skew.AdvectionModel(a), "skew")
    assert abs(ent) < 1e-13 * scale
    ent_up, scale_up = energy_rate(skew.AdvectionModel(a, upwind=True), "skew")
    assert ent_up < -1e-3 * scale_up
    if p >= 3:
        ent_cons, scale_cons = energy_rate(skew.AdvectionModel(a), "cons")
        assert abs(ent_cons) > 1e-8 * scale_cons


@pytest.mark.parametrize("dim,M,p", [(2, 3, 3), (3, 3, 2)])
def test_skew_volume_term_is_a_line_pair_sum(dim, M, p):
    """The volume term of Eq. (rhs_skew) equals sum_j sum_m c^m_ij f_m(u_j) with
    c^m_ij = 1/2 sum_l (Q^(l)_ji G_lm(j) - G_lm(i) Q^(l)_ij), and c^m_ij vanishes unless i
    and j lie on a common collapsed-coordinate line (the sparsity of Q^(l), Section 5.1)."""
    D = disc(dim, M, p, True)
    um = euler_state(D, 11)
    model = skew.EulerModel(dim)
    u, _ = skew.nodal_states(D, um)
    e = 4
    G = D.geo.G_vol[e]
    f = [model.flux(u[e], m) for m in range(dim)]
    vol = sum(0.5 * (D.ref.Q[l].T @ (G[:, l, m][:, None] * f[m]) - G[:, l, m][:, None] * (D.ref.Q[l] @ f[m]))
              for l in range(dim) for m in range(dim))
    alpha = D.ref.alpha
    same_line = (alpha[:, None, :] == alpha[None, :, :]).sum(-1) >= dim - 1
    pair = np.zeros_like(vol)
    for m in range(dim):
        c = sum(0.5 * (D.ref.Q[l].T * G[None, :, l, m] - G[:, l, m][:, None] * D.ref.Q[l]) for l in range(dim))
        assert np.all(c[~same_line] == 0.0)
        assert np.allclose(np.diag(c), 0.0, atol=1e-13 * np.abs(c).max())
        pair += c @ f[m]
    assert np.abs(pair - vol).max() < 1e-13 * np.abs(vol).max()


def test_skew_form_in_long_double_matches_fp64():
    """The skew-symmetric form evaluated in long double on a sub-mesh agrees with FP64 to FP64
    rounding, and its free-stream residual vanishes to long-double rounding (Euler, curved
    tetrahedra): the extended-precision reference the GPU tests use."""
    from oracle import extended
    X = np.longdouble
    if np.finfo(X).eps >= np.finfo(float).eps / 100:
        pytest.skip("no extended long double")
    L = 2 * np.pi
    mesh, Xn = I.config_mesh(3, 3, L, 2, True)
    D = Discretization(3, 2, Xn, mesh.nbr_elem, mesh.nbr_face)
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, I.density_wave(D.geo.x_vol, L))
    el = np.array([3, 50])
    Dx, need, local = extended.sub_discretization(3, 2, Xn, mesh.nbr_elem, mesh.nbr_face, el)
    model = skew.EulerModel(3)
    rx = skew.rhs(Dx, um[need].astype(X), model, "skew", local)
    r64 = skew.rhs(D, um, model, "skew", el)
    assert rx.dtype == X
    assert np.abs(rx - r64).max() < 1e-12 * np.abs(rx).max()
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7, 0.2]), np.array(2.1))
    uc = np.zeros((D.E, 5, D.Np))
    uc[:, :, 0] = ubar / D.V[0, 0]
    rf = skew.rhs(Dx, uc[need].astype(X), model, "skew", local)
    assert np.abs(rf).max() < 1e4 * np.finfo(X).eps * np.abs(ubar).max()
