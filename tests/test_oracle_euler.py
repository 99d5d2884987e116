"""Pins for the oracle's Euler physics (Section 7.1-7.2, Definitions 1, 5, 6)."""
import numpy as np
import pytest
from mpmath import mp, mpf, log as mlog

from oracle import euler

RNG = np.random.default_rng(1234)


def random_states(n, d, rng=RNG):
    rho = rng.uniform(0.3, 3.0, n)
    v = rng.normal(0, 1.0, (n, d))
    p = rng.uniform(0.2, 5.0, n)
    return euler.conservative(rho, v, p)


def cs_grad(f, U, h=1e-30):
    """Complex-step gradient of a scalar function of the state (exact to rounding)."""
    out = np.zeros(U.shape)
    for k in range(U.shape[-1]):
        Uc = U.astype(complex)
        Uc[..., k] += 1j * h
        out[..., k] = np.imag(f(Uc)) / h
    return out


@pytest.mark.parametrize("d", [2, 3])
def test_entropy_variables_are_gradient(d):
    U = random_states(50, d)
    g = cs_grad(euler.entropy, U)
    assert np.allclose(euler.entropy_vars(U), g, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_entropy_flux_pair(d):
    """(grad F_m)^T = (grad S)^T grad f_m  (Eq. (entropy_contract))."""
    U = random_states(20, d)
    w = euler.entropy_vars(U)
    for m in range(d):
        gF = cs_grad(lambda X: euler.entropy_flux(X, m), U)
        for i in range(len(U)):
            Jf = np.stack([np.imag(euler.euler_flux(U[i].astype(complex) + 1j * 1e-30 * np.eye(d + 2)[k], m)) / 1e-30
                           for k in range(d + 2)], axis=1)
            assert np.allclose(gF[i], w[i] @ Jf, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_inverse_entropy_map(d):
    U = random_states(200, d)
    assert np.allclose(euler.cons_from_entropy(euler.entropy_vars(U)), U, rtol=1e-13, atol=1e-13)


def test_log_mean_against_high_precision():
    mp.dps = 40
    a = RNG.uniform(0.1, 10, 400)
    rel = np.concatenate([RNG.uniform(-1e-3, 1e-3, 200), RNG.uniform(-0.9, 3, 200)])
    b = a * (1 + rel)
    lm = euler.log_mean(a, b)
    ilm = euler.inv_log_mean(a, b)
    for i in range(len(a)):
        A, B = mpf(a[i]), mpf(b[i])
        exact = (B - A) / (mlog(B) - mlog(A)) if A != B else A
        # forward error model of the direct branch: the rounded ratio b/a perturbs ln(b/a)
        # by ~eps absolutely, i.e. by eps/|ln(b/a)| relatively
        tol = 4 * np.finfo(float).eps * (1 + 1 / abs(np.log(b[i] / a[i])))
        assert abs(float((mpf(lm[i]) - exact) / exact)) < tol
        assert abs(float((mpf(ilm[i]) - 1 / exact) * exact)) < tol
    assert np.all(euler.log_mean(a, a) == a) or np.allclose(euler.log_mean(a, a), a, rtol=2e-16)


@pytest.mark.parametrize("d", [2, 3])
def test_ranocha_flux_consistent_symmetric(d):
    """Definition 5: symmetric and consistent, f_m^#(U,U) = f_m(U)."""
    UL, UR = random_states(100, d), random_states(100, d)
    for m in range(d):
        assert np.allclose(euler.ranocha_flux(UL, UR, m), euler.ranocha_flux(UR, UL, m), rtol=1e-14, atol=1e-14)
        assert np.allclose(euler.ranocha_flux(UL, UL, m), euler.euler_flux(UL, m), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_tadmor_shuffle_condition(d):
    """Eq. (tadmor) with Psi_m = W^T f_m - F_m computed from the definitions (Section 2.2)."""
    UL, UR = random_states(2000, d), random_states(2000, d)
    UR[:1000] = UL[:1000] * (1 + RNG.uniform(-1e-3, 1e-3, (1000, 1)))   # nearly equal states too
    wL, wR = euler.entropy_vars(UL), euler.entropy_vars(UR)
    for m in range(d):
        psiL = np.sum(wL * euler.euler_flux(UL, m), -1) - euler.entropy_flux(UL, m)
        psiR = np.sum(wR * euler.euler_flux(UR, m), -1) - euler.entropy_flux(UR, m)
        F = euler.ranocha_flux(UL, UR, m)
        lhs = np.sum((wR - wL) * F, -1)
        # rounding scale of both sides (w^+ - w^- cancels for nearly equal states)
        scale = (np.abs(wR * F).sum(-1) + np.abs(wL * F).sum(-1) + np.abs(psiR) + np.abs(psiL))
        assert np.max(np.abs(lhs - (psiR - psiL)) / scale) < 1e-14


def test_printed_energy_term_would_fail_consistency():
    """The energy component exactly as printed (1/2 on both terms) is not consistent; the
    oracle's reading is (this is the reading recorded for Eq. (ranocha_flux))."""
    U = random_states(10, 3)
    rho, v, p = euler.primitive(U)
    m = 0
    printed = 0.5 * rho * v[:, m] * (np.sum(v * v, -1) + 1 / (euler.GAMMA - 1) * p / rho) + p * v[:, m]
    exact = euler.euler_flux(U, m)[:, -1]
    assert np.max(np.abs(printed - exact) / np.abs(exact)) > 1e-2
    assert np.allclose(euler.ranocha_flux(U, U, m)[:, -1], exact, rtol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_interface_flux_properties(d):
    """Definition 6: conservation, consistency, and the entropy condition Eq. (tadmor_directional)."""
    UL, UR = random_states(500, d), random_states(500, d)
    n = RNG.normal(size=(500, d)); n /= np.linalg.norm(n, axis=1, keepdims=True)
    for diss in (False, True):
        f = euler.interface_flux(UL, UR, n, diss)
        assert np.allclose(f, -euler.interface_flux(UR, UL, -n, diss), rtol=1e-13, atol=1e-13)
        assert np.allclose(euler.interface_flux(UL, UL, n, diss), euler.euler_flux_dir(UL, n), rtol=1e-13, atol=1e-13)
        wL, wR = euler.entropy_vars(UL), euler.entropy_vars(UR)
        psi = lambda U, w: np.stack([np.sum(w * euler.euler_flux(U, m), -1) - euler.entropy_flux(U, m) for m in range(d)], -1)
        lhs = np.sum((wR - wL) * f, -1)
        rhs = np.sum((psi(UR, wR) - psi(UL, wL)) * n, -1)
        scale = (np.abs(wR * f).sum(-1) + np.abs(wL * f).sum(-1)
                 + np.abs(psi(UR, wR)).sum(-1) + np.abs(psi(UL, wL)).sum(-1))
        if diss:
            assert np.all(lhs - rhs <= 1e-12 * scale)
            assert np.mean(lhs - rhs < -1e-6 * scale) > 0.9
        else:
            assert np.max(np.abs(lhs - rhs) / scale) < 1e-13


def test_davis_speed_closed_form():
    U = euler.conservative(np.array([1.0]), np.array([[3.0, -4.0]]), np.array([1.0 / 1.4]))
    V = euler.conservative(np.array([4.0]), np.array([[0.0, 1.0]]), np.array([1.4 * 4 / 1.4]))
    n = np.array([[0.6, 0.8]])
    # |vL.n| = |1.8-3.2| = 1.4, |vR.n| = 0.8; cL = 1, cR = sqrt(1.4*4/4)= sqrt(1.4)
    assert np.allclose(euler.davis_speed(U, V, n), 1.4 + np.sqrt(1.4))
