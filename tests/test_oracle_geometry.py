"""Pins for the oracle's geometry (Sections 4.1, 4.2, 4.5, 6: Eq. (poly_mapping),
Eq. (metric_identities), Eq. (conservative_curl), Eq. (nanson), Eq. (jacobian_approx))."""
from functools import lru_cache

import numpy as np
import pytest

import esd_inputs as I
from oracle.reference import RefElement
from oracle.geometry import Geometry, lagrange_simplex, lattice


@lru_cache(maxsize=None)
def build(dim, M, p, warp, L=2 * np.pi):
    mesh, X = I.config_mesh(dim, M, L, p, warp)
    ref = RefElement(dim, p)
    return mesh, X, ref, Geometry(ref, X, mesh.nbr_elem, mesh.nbr_face)


def adjugate(A):
    """G_lm = J d xi_l/d x_m from the Jacobian A[m, l] = d x_m / d xi_l."""
    return np.linalg.det(A)[..., None, None] * np.linalg.inv(A)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 3), (3, 1), (3, 2), (3, 4)])
def test_affine_metrics_closed_form(dim, p):
    mesh, X, ref, g = build(dim, 3, p, False)
    # affine map: d x / d xi = (v_{k+1} - v_1)/2 (column k)
    A = 0.5 * np.transpose(mesh.verts[:, 1:, :] - mesh.verts[:, :1, :], (0, 2, 1))
    Gex = adjugate(A)
    assert np.abs(g.G_vol - Gex[:, None]).max() < 1e-12
    for z in range(ref.Nf):
        assert np.abs(g.G_fac[z] - Gex[:, None]).max() < 1e-12
    assert np.abs(g.J_vol - np.linalg.det(A)[:, None]).max() < 1e-12
    # outward unit normals: orthogonal to the facet's edges, pointing away from the opposite vertex
    for z, loc in enumerate(I.LOCAL_FACETS[dim]):
        v = mesh.verts
        opp = [k for k in range(dim + 1) if k not in loc][0]
        n = g.n_fac[z][:, 0]
        for k in loc[1:]:
            assert np.abs(np.sum(n * (v[:, k] - v[:, loc[0]]), -1)).max() < 1e-12
        assert np.all(np.sum(n * (v[:, opp] - v[:, loc[0]]), -1) < 0)


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2), (3, 3), (3, 4)])
def test_discrete_metric_identities(dim, p):
    """sum_l D^(l) G_lm = 0 at the volume nodes (Eq. (metric_identities) with G in P_q)."""
    mesh, X, ref, g = build(dim, 3, p, True)
    for m in range(dim):
        res = sum(np.einsum("ij,ej->ei", ref.D[l], g.G_vol[:, :, l, m]) for l in range(dim))
        assert np.abs(res).max() < 1e-12 * np.abs(g.G_vol).max() * p ** 2


@pytest.mark.parametrize("p", [1, 2])
def test_curl_form_equals_adjugate_when_interpolation_exact(p):
    """For an isoparametric map with 2 p_g - 1 <= q + 1 the curl form is the exact adjugate."""
    mesh, X, ref, g = build(3, 3, p, True)
    pts = np.concatenate([ref.xi] + ref.xif)
    _, dL = lagrange_simplex(3, p, pts)
    A = np.einsum("tik,eim->etmk", dL, X)
    assert np.abs(g.G_all - adjugate(A)).max() < 1e-11


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_watertight_volume(dim, p):
    """Conforming curved elements tile the periodic box: sum of int det(grad x) = L^d
    (quadrature exact for det of degree d(p_g-1) <= 2q)."""
    L = 2 * np.pi
    mesh, X, ref, g = build(dim, 3, p, True)
    assert abs(np.sum(ref.w * g.J_exact_vol) - L ** dim) < 1e-11 * L ** dim
    assert np.all(g.J_vol > 0)


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2), (3, 3)])
def test_interpolated_jacobian(dim, p):
    """J of Eq. (jacobian_approx) interpolates det(grad x) at the mapping nodes."""
    mesh, X, ref, g = build(dim, 3, p, True)
    lat = lattice(dim, p)
    L, dL = lagrange_simplex(dim, p, lat)
    assert np.abs(L - np.eye(len(lat))).max() < 1e-11
    A = np.einsum("tik,eim->etmk", dL, X)
    assert np.abs(g.det_lattice - np.linalg.det(A)).max() < 1e-12


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2), (3, 4)])
def test_facet_matching(dim, p):
    """Assumption 2: matched facet nodes coincide (up to the periodic shift), normals are
    opposite and omega J^(kappa,zeta) agree."""
    mesh, X, ref, g = build(dim, 3, p, True)
    for e in range(g.E):
        for z in range(ref.Nf):
            e2, z2 = mesh.nbr_elem[e, z], mesh.nbr_face[e, z]
            P = g.perm[e, z]
            d = g.x_fac[z][e] - g.x_fac[z2][e2][P]
            shift = np.round(d[0] / mesh.L) * mesh.L
            assert np.abs(d - shift).max() < 1e-12
            assert np.abs(g.n_fac[z][e] + g.n_fac[z2][e2][P]).max() < 1e-12
            assert np.abs(ref.wf[z] * g.Jf[z][e] - ref.wf[z2][P] * g.Jf[z2][e2][P]).max() < 1e-12
