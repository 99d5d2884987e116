"""Conservation and entropy over a run (the long-run monitoring of Section 7.5): the
totals of esd_integrals against the oracle's quadrature, and their time series over RK4
steps -- conserved totals constant to rounding, total entropy constant to the time
integration error with the entropy-conservative flux and non-increasing with
Lax-Friedrichs dissipation, entropy rate zero to rounding (EC) at every sample."""
import numpy as np
import pytest

import esd_inputs as I
from oracle import euler
from gpu_common import workload, gpu_mesh, to_dev

pytestmark = pytest.mark.gpu


def oracle_totals(D, um):
    """sum over elements of W J (V u~) per variable and of W J S(V u~)."""
    u = D.to_nodal(um)                                  # [E, Nq, Nc]
    wj = D.ref.w[None, :] * D.geo.J_vol                 # [E, Nq]
    return np.concatenate([np.einsum("ei,eic->c", wj, u), [np.sum(wj * euler.entropy(u))]])


@pytest.mark.parametrize("dim,M,p,state", [(2, 4, 3, "vortex"), (3, 3, 3, "tgv"), (3, 3, 2, "density_wave")])
def test_integrals_match_oracle(dim, M, p, state):
    mesh, X, D, um = workload(dim, M, p, True, "LF", state)
    gm = gpu_mesh(dim, p, X, mesh)
    got = gm.integrals(to_dev(um)).cpu().numpy()
    ref = oracle_totals(D, um)
    scale = np.abs(ref) + 1e-300
    assert np.all(np.abs(got - ref) <= 1e-13 * np.maximum(scale, np.abs(ref).max() * 1e-3)), (got, ref)


@pytest.mark.parametrize("flux", ["EC", "LF"])
def test_time_series_conservation_and_entropy(flux):
    mesh, X, D, um = workload(3, 3, 3, True, flux, "tgv")
    gm = gpu_mesh(3, 3, X, mesh, flux)
    L = 2 * np.pi
    lam = I.max_wave_speed_sampled(I.config_state_fn(3, L, "tgv"), 3, L)
    dt = 0.1 * (L / 3) / (lam * 7)
    steps, tot, rates = gm.run_diagnostics(to_dev(um), dt, 40, every=5)
    nc = 5
    # conserved totals: constant up to rounding (RK4 keeps linear invariants)
    drift = np.abs(tot[:, :nc] - tot[0, :nc]).max(axis=0)
    scale = np.abs(tot[0, :nc]).max()
    assert np.all(drift <= 1e-12 * scale), (drift, scale)
    # rates of the conserved variables (Theorem 2): zero to rounding at every sample
    assert np.all(np.abs(rates[:, :nc]) <= 1e-11 * np.abs(tot[0, :nc]).max())
    S = tot[:, nc]
    if flux == "EC":
        # entropy rate zero to rounding at every sample (Theorem 4); total entropy constant
        # up to the time integration error
        assert np.all(np.abs(rates[:, nc]) <= 1e-12 * rates[:, nc + 1]), rates[:, nc:]
        assert np.abs(S - S[0]).max() <= 1e-9 * np.abs(S[0]), S
    else:
        # dissipation: the entropy rate is non-positive and the total entropy does not grow
        assert np.all(rates[:, nc] <= 1e-12 * rates[:, nc + 1]), rates[:, nc:]
        assert np.all(np.diff(S) <= 1e-12 * np.abs(S[0])), np.diff(S)
