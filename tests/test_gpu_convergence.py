"""Accuracy of the whole GPU path against an exact solution: the density wave of Section
7.4 (rho = 1 + sin(2 pi sum(x)/L)/5, v = 1, p = 1) is advected without change of shape, so
after time T the exact state is the initial one shifted by T in every coordinate.  The
L2 error of the density (quadrature of the mass matrix) on curved meshes refined by 2
must fall at a rate near the optimal p + 1 for the Lax-Friedrichs interface flux: the test
asks for at least p + 1/2 between the two finest meshes."""
import math

import numpy as np
import pytest

import esd_inputs as I
from oracle.residual import Discretization
from gpu_common import gpu_mesh, to_dev

pytestmark = pytest.mark.gpu

L = 2.0
T = 0.2


def density_error(dim, M, p):
    mesh, X = I.config_mesh(dim, M, L, p, True)
    D = Discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux="LF")
    f0 = lambda x: I.density_wave(x, L)                                   # noqa: E731
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, f0(D.geo.x_vol))     # reference L2 projection
    gm = gpu_mesh(dim, p, X, mesh, "LF")
    lam = I.max_wave_speed_sampled(f0, dim, L)
    n = math.ceil(T / (0.05 * (L / M) / (lam * (2 * p + 1))))
    dt = T / n
    u = to_dev(um)
    for _ in range(n):
        gm.rk_step(u, dt)
    gm.check()
    rho_h = D.to_nodal(u.cpu().numpy())[..., 0]
    rho_ex = f0(D.geo.x_vol - T)[..., 0]
    wj = D.ref.w[None, :] * D.geo.J_vol
    return math.sqrt(np.sum(wj * (rho_h - rho_ex) ** 2))


@pytest.mark.parametrize("dim,p,Ms", [(2, 2, (4, 8, 16)), (2, 3, (4, 8, 16)), (3, 2, (4, 8, 12))])
def test_density_wave_convergence(dim, p, Ms):
    errs = [density_error(dim, M, p) for M in Ms]
    rates = [math.log(a / b) / math.log(mb / ma) for a, b, ma, mb in zip(errs, errs[1:], Ms, Ms[1:])]
    print(f"density wave dim={dim} p={p} M={Ms}: L2 errors {errs}, rates {rates}")
    assert errs[-1] < errs[0]
    assert rates[-1] >= p + 0.5, (errs, rates)
