"""The differentiation workload at its full size: the VJP of esd_rhs on 8^3 x 6 = 3072
curved tetrahedra at p = 3 (Taylor-Green state at Mach 0.1 plus seeded N(0, 1e-3) on every
mode, cotangent N(0, 1)), checked per element against the oracle's complex-step Jacobian
transpose on sampled elements and as a whole against central differences of the GPU
forward; and the 20-step RK4 rollout with per-stage checkpoints through torch.autograd
against central differences."""
from functools import lru_cache

import numpy as np
import pytest

import esd_inputs as I
from oracle.residual import Discretization
from gpu_common import gpu_mesh, to_dev, check_vjp_parity, periodic_face_elements

pytestmark = pytest.mark.gpu

L = 2 * np.pi


@lru_cache(maxsize=None)
def case(flux):
    mesh, X = I.config_mesh(3, 8, L, 3, True)
    D = Discretization(3, 3, X, mesh.nbr_elem, mesh.nbr_face, flux=flux)
    f = I.config_state_fn(3, L, "tgv")
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, f(D.geo.x_vol)) + I.seeded_normal(21, (D.E, D.Nc, D.Np), 1e-3)
    cot = I.seeded_normal(22, um.shape, 1.0)
    return mesh, X, D, np.ascontiguousarray(um), cot


@pytest.mark.parametrize("flux", ["LF", "EC"])
def test_vjp_fullsize_per_element_against_oracle(flux):
    """Element-wise (J^T c) on 8 sampled elements, 4 of them with a facet across the
    periodic boundary, against the oracle's complex-step Jacobian transpose in FP64 and in
    long double (criteria of gpu_common.check_vjp_parity)."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um, cot = case(flux)
    gm = gpu_mesh(3, 3, X, mesh, flux)
    g = torch.empty((D.E, D.Nc, D.Np), dtype=torch.float64, device="cuda")
    E.esd_rhs_vjp(gm.handle, to_dev(um), to_dev(cot), g)
    g = g.cpu().numpy()
    gm.check()
    rng = np.random.default_rng(23)
    per = periodic_face_elements(mesh)
    inner = np.setdiff1d(np.arange(D.E), per)
    sample = np.concatenate([rng.choice(per, 4, replace=False), rng.choice(inner, 4, replace=False)])
    check_vjp_parity(f"vjp full-size 3072 tets p=3 tgv {flux}", g, D, X, um, cot, sample)


@pytest.mark.parametrize("flux,h", [("EC", 1e-6), ("LF", 1e-7)])
def test_vjp_fullsize_central_differences(flux, h):
    """<c, (R(u + h v) - R(u - h v)) / 2h> (Richardson of h, 2h) against <J^T c, v>.  The LF
    dissipation's max/|.| kinks lie within ~1e-6 of a smooth state, hence h = 1e-7 there."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um, cot = case(flux)
    gm = gpu_mesh(3, 3, X, mesh, flux)
    u, c = to_dev(um), to_dev(cot)
    v = to_dev(I.seeded_normal(24, um.shape, 1.0))

    def cd(hh):
        return (gm.rhs(u + hh * v) - gm.rhs(u - hh * v)) / (2 * hh)
    fd = (4.0 * cd(h) - cd(2 * h)) / 3.0
    g = torch.empty_like(u)
    E.esd_rhs_vjp(gm.handle, u, c, g)
    lhs, rhs = float((c * fd).sum()), float((g * v).sum())
    assert abs(lhs - rhs) < 1e-6 * float((c * fd).abs().sum()), (lhs, rhs)


def test_rollout_fullsize_central_differences():
    """20 RK4 steps at CFL 0.1 with per-stage checkpoints: d<w, u_20>/du_0 . v against
    Richardson-extrapolated central differences with h = 1e-6 (entropy-conservative flux,
    smooth in the state)."""
    import torch
    from paper_2312_07874_gb300.autograd import rollout
    mesh, X, D, um, cot = case("EC")
    gm = gpu_mesh(3, 3, X, mesh, "EC")
    lam = I.max_wave_speed_sampled(I.config_state_fn(3, L, "tgv"), 3, L)
    dt = 0.1 * (L / 8) / (lam * 7)
    w = to_dev(cot)
    v = to_dev(I.seeded_normal(25, um.shape, 1.0))
    u0 = to_dev(um).requires_grad_(True)
    (w * rollout(u0, gm, dt, 20, "stages")).sum().backward()
    ad = float((u0.grad * v).sum())

    def loss(x):
        with torch.no_grad():
            return float((w * rollout(x, gm, dt, 20, "stages")).sum())

    def cd(hh):
        return (loss(to_dev(um) + hh * v) - loss(to_dev(um) - hh * v)) / (2 * hh)
    fd = (4.0 * cd(1e-6) - cd(2e-6)) / 3.0
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)
