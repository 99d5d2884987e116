"""Pins for the oracle's residual (Sections 4.4-4.6, 5, 6): three independent routes agree,
and the discretisation satisfies the theorems of Section 6 to rounding."""
from functools import lru_cache

import numpy as np
import pytest

import esd_inputs as I
from oracle import euler
from oracle.residual import Discretization
from oracle.timestep import rk4_step


@lru_cache(maxsize=None)
def disc(dim, M, p, warp, flux, state):
    L = 2 * np.pi
    mesh, X = I.config_mesh(dim, M, L, p, warp)
    D = Discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux=flux)
    f = I.config_state_fn(dim, L, state)
    u0 = f(D.geo.x_vol)
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, u0)
    um = um + I.seeded_normal(7, um.shape, 1e-3)
    return D, um


CASES = [(2, 3, p, w, f, "vortex") for p in (1, 2, 4) for w in (False, True) for f in ("EC", "LF")] + \
        [(3, 3, p, True, f, "tgv") for p in (1, 2) for f in ("EC", "LF")]


@pytest.mark.parametrize("case", CASES)
def test_three_routes_agree(case):
    D, um = disc(*case)
    el = np.arange(min(D.E, 12))
    a = D.rhs(um, "dense", elems=el)
    b = D.rhs(um, "sparse", elems=el)
    c = D.rhs_hybridized(um, elems=el)
    scale = np.abs(a).max()
    assert np.abs(a - b).max() < 1e-13 * scale
    assert np.abs(a - c).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_free_stream(dim, p):
    """Theorem 3: a uniform state has zero time derivative on curved periodic meshes."""
    D, _ = disc(dim, 3, p, True, "LF", "vortex" if dim == 2 else "tgv")
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7, 0.2][:dim]), np.array(2.1))
    un = np.broadcast_to(ubar, (D.E, D.ref.Nq, D.Nc))
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, un)
    el = np.arange(min(D.E, 20))
    r = D.rhs(um, "sparse", elems=el)
    assert np.abs(r).max() < 1e-12 * np.abs(ubar).max()


@pytest.mark.parametrize("case", [(2, 3, 3, True, "LF", "vortex"), (3, 3, 2, True, "LF", "tgv"),
                                  (3, 3, 3, True, "EC", "tgv")])
def test_conservation(case):
    """Theorem 2: sum_kappa 1^T W J V d u~/dt = 0 on periodic meshes."""
    D, um = disc(*case)
    dudt = D.rhs(um, "sparse")
    rate = D.conservation_rate(dudt)
    y = np.einsum("ij,ecj->eic", D.V, dudt)
    scale = np.einsum("i,ei,eic->c", D.ref.w, D.geo.J_vol, np.abs(y))
    assert np.all(np.abs(rate) < 1e-13 * scale)


@pytest.mark.parametrize("dim,M,p,state", [(2, 3, 2, "vortex"), (2, 3, 4, "vortex"), (3, 3, 2, "tgv"),
                                           (3, 3, 3, "tgv")])
def test_entropy_conservation_and_stability(dim, M, p, state):
    """Theorem 4: entropy rate = 0 with the EC interface flux and <= 0 with LF (to 1e-12 relative)."""
    D, um = disc(dim, M, p, True, "EC", state)
    ent, scale = D.entropy_rate(um, D.rhs(um, "sparse"))
    assert abs(ent) < 1e-12 * scale
    D2, um2 = disc(dim, M, p, True, "LF", state)
    ent2, scale2 = D2.entropy_rate(um2, D2.rhs(um2, "sparse"))
    assert ent2 < 1e-12 * scale2
    assert ent2 < -1e-8 * scale2          # the dissipation is actually active for this state


def test_affine_projection_is_l2_projection():
    """With constant J the weight-adjusted entropy projection is V^T W W(V u~)."""
    D, um = disc(2, 3, 3, False, "LF", "vortex")
    wt = D.project_entropy(um)
    direct = np.einsum("ij,i,eic->ejc", D.V, D.ref.w, euler.entropy_vars(D.to_nodal(um)))
    assert np.abs(wt - direct).max() < 1e-13 * np.abs(direct).max()


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_sparse_route_flux_count(dim, p):
    """The paper's algorithm evaluates exactly Eq. (num_fluxes) fluxes per element."""
    D, um = disc(dim, 3, p, True, "LF", "vortex" if dim == 2 else "tgv")
    _, count = D.nodal_residual(um, "sparse", elems=np.arange(1), return_count=True)
    q = p
    expect = 1.5 * (q + 1) ** 2 * (q + 2) if dim == 2 else 4 * (q + 1) ** 4
    assert count == expect


def test_planted_mistakes_are_caught():
    """Mistakes planted in the oracle (on the CPU) break a pin: dropping the facet correction
    breaks free-stream preservation; a sign error in C^T 1 breaks entropy conservation."""
    D, um = disc(2, 3, 2, True, "EC", "vortex")
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7]), np.array(2.1))
    uf = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, np.broadcast_to(ubar, (D.E, D.ref.Nq, D.Nc)))
    orig = D._residual_dense

    # (1) drop the correction: use the skew-free volume term plus plain lift
    def dropped(el, Ut, Utf, fstar):
        ref, geo, d = D.ref, D.geo, D.dim
        U, G = Ut[el], geo.G_vol[el]
        F = [euler.ranocha_flux(U[:, :, None, :], U[:, None, :, :], m) for m in range(d)]
        r = np.zeros(U.shape)
        for l in range(d):
            acc = sum(0.5 * (G[:, :, None, l, m] + G[:, None, :, l, m])[..., None] * F[m] for m in range(d))
            r -= np.einsum("ij,eijc->eic", 2.0 * ref.S[l], acc)
        for z in range(ref.Nf):
            g = (ref.wf[z][None, :] * geo.Jf[z][el])[..., None] * fstar[z]
            r -= np.einsum("ji,ejc->eic", ref.R[z], g)
        return r
    D._residual_dense = dropped
    try:
        assert np.abs(D.rhs(uf, "dense", elems=np.arange(4))).max() > 1e-6
    finally:
        D._residual_dense = orig

    # (2) sign error in the C^T 1 term
    def flipped(el, Ut, Utf, fstar):
        ref, geo, d = D.ref, D.geo, D.dim
        U, G = Ut[el], geo.G_vol[el]
        r = dropped(el, Ut, Utf, fstar)
        for z in range(ref.Nf):
            Uf = Utf[z][el]
            JnV = np.einsum("eilm,l->eim", G, ref.nhat[z])
            JnF = geo.Jn_fac[z][el]
            Ff = [euler.ranocha_flux(U[:, :, None, :], Uf[:, None, :, :], m) for m in range(d)]
            acc = sum(0.5 * (JnV[:, :, None, m] + JnF[:, None, :, m])[..., None] * Ff[m] for m in range(d))
            C = (ref.R[z].T @ ref.B[z])[None, :, :, None] * acc
            r -= C.sum(axis=2) + np.einsum("ji,ejc->eic", ref.R[z], C.sum(axis=1))   # wrong sign
        return r
    D._residual_dense = flipped
    try:
        ent, scale = D.entropy_rate(um, D.rhs(um, "dense"))
        assert abs(ent) > 1e-6 * scale
    finally:
        D._residual_dense = orig


def test_rk4_fourth_order():
    lam = -0.7 + 0.3j
    f = lambda u: lam * u
    errs = []
    for n in (10, 20, 40):
        u, dt = 1.0 + 0j, 1.0 / n
        for _ in range(n):
            u = rk4_step(f, u, dt)
        errs.append(abs(u - np.exp(lam)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8)


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_weight_adjusted_inverse_exact_on_polynomials(dim, p):
    """Eq. (weight_adjusted_inverse): M~^-1 = V^T W J^-1 V inverts M_J = V^T W J V exactly on
    modes c whenever J (V c) is a polynomial of degree <= p (the quadrature is exact to degree
    2q), and only approximately otherwise.  J is planted as a positive affine function of xi."""
    import copy
    from oracle.pkd import modal_indices
    D, _ = disc(dim, 3, p, True, "LF", "vortex" if dim == 2 else "tgv")
    Dp = copy.copy(D)
    Dp.geo = copy.copy(D.geo)
    xi = D.ref.xi
    J = 2.0 + xi @ np.array([0.3, -0.2, 0.1][:dim])
    Dp.geo.J_vol = np.broadcast_to(J, (D.E, D.ref.Nq))
    deg = np.array([sum(a) for a in modal_indices(dim, p)])
    rng = np.random.default_rng(11)
    c = rng.standard_normal((1, D.Np, D.Nc))
    low = np.where(deg <= p - 1, 1.0, 0.0)[None, :, None] * c
    MJ = lambda y: np.einsum("qi,q,qk,ekc->eic", D.V, D.ref.w * J, D.V, y)
    assert np.abs(Dp.minv(MJ(low), np.arange(1)) - low).max() < 1e-13 * np.abs(low).max()
    assert np.abs(Dp.minv(MJ(c), np.arange(1)) - c).max() > 1e-6 * np.abs(c).max()
    # constant J: the weight-adjusted inverse is exactly M_J^-1 = I / J on every mode
    Dp.geo.J_vol = np.full((D.E, D.ref.Nq), 1.7)
    assert np.abs(Dp.minv(1.7 * c, np.arange(1)) - c).max() < 1e-13 * np.abs(c).max()
