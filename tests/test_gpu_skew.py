"""The skew-symmetric form on the GPU (esd_rhs_skew, Eq. (rhs_skew)) against the oracle's
skew-symmetric form (oracle/skew.py), for the compressible Euler equations and for scalar
linear advection, element by element on small curved meshes (several tiles and a ragged
last tile, every degree class).  Criteria as for the entropy-stable residual
(gpu_common): accuracy against the oracle in long double within 10 x the FP64 oracle's own
error, and the 1e-12 parity target against long double where an FP64 evaluation reaches it."""
import numpy as np
import pytest

import esd_inputs as I
from gpu_common import to_dev, rel_err_per_var, C_EXACT, FLOOR, FLAT_REACH, PARITY_TOL, _log
from oracle import extended, skew
from oracle.residual import Discretization

pytestmark = pytest.mark.gpu
L = 2 * np.pi
A = (1.0, 0.6, -0.35)


def setup(dim, M, p, model, state, flux="LF", upwind=False, seed=0):
    import paper_2312_07874_gb300 as E
    mesh, X = I.config_mesh(dim, M, L, p, True)
    D = Discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux=flux)
    if model == "euler":
        u0 = I.config_state_fn(dim, L, state)(D.geo.x_vol)
        om = skew.EulerModel(dim, dissipation=(flux == "LF"))
    else:   # a smooth scalar: the density of the density wave
        u0 = I.density_wave(D.geo.x_vol, L)[..., :1]
        om = skew.AdvectionModel(A[:dim], upwind=upwind)
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, u0)
    um = np.ascontiguousarray(um + I.seeded_normal(90 + seed, um.shape, 1e-3))
    gs = E.Skew(dim, p, X, mesh.nbr_elem, mesh.nbr_face, model=model, a=A[:dim], upwind=upwind, flux=flux)
    return mesh, X, D, um, om, gs


def check(label, got, D, X, mesh, um, om, n_exact=3, seed=0):
    """Element-wise against the FP64 skew oracle on every element, and against the skew
    oracle in long double on a sample."""
    ref = skew.rhs(D, um, om, "skew")
    e_flat = np.asarray(rel_err_per_var(got, ref), dtype=float)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(D.E, size=n_exact, replace=False))
    Dx, need, local = extended.sub_discretization(D.dim, D.p, X, mesh.nbr_elem, mesh.nbr_face, pick,
                                                  flux="LF" if D.dissipation else "EC")
    rx = skew.rhs(Dx, um[need].astype(extended.EXT), om, "skew", local)
    e_gpu = np.asarray(rel_err_per_var(got[pick], rx), dtype=float)
    e_64 = np.asarray(rel_err_per_var(ref[pick], rx), dtype=float)
    flat = e_64 < FLAT_REACH
    rec = dict(case=label, e_gpu_exact=e_gpu.tolist(), e_oracle64_exact=e_64.tolist(),
               e_gpu_oracle64=e_flat.tolist(), flat=flat.tolist(), n_elems=int(D.E), n_exact=int(len(pick)))
    _log(rec)
    print(rec)
    assert np.all(e_gpu <= C_EXACT * np.maximum(e_64, FLOOR)), ("accuracy vs exact", label, e_gpu, e_64)
    assert np.all(e_gpu[flat] < PARITY_TOL), ("flat bound vs exact", label, e_gpu, e_64)
    # a gross defect anywhere (a dropped or mis-signed term) is O(1) against the FP64 oracle
    assert np.all(e_flat < 1e-9), ("against the FP64 oracle", label, e_flat)


EULER_CASES = [(2, 3, 1, "vortex"), (2, 4, 2, "vortex"), (2, 3, 4, "vortex"), (2, 3, 7, "vortex"),
               (2, 3, 10, "vortex"), (3, 3, 1, "density_wave"), (3, 3, 2, "density_wave"),
               (3, 3, 3, "density_wave"), (3, 3, 4, "density_wave"), (3, 3, 2, "tgv"), (3, 3, 6, "density_wave")]


@pytest.mark.parametrize("dim,M,p,state", EULER_CASES)
@pytest.mark.parametrize("flux", ["LF", "EC"])
def test_skew_euler_parity(dim, M, p, state, flux):
    import torch
    mesh, X, D, um, om, gs = setup(dim, M, p, "euler", state, flux, seed=p)
    out = gs.rhs(to_dev(um))
    torch.cuda.synchronize()
    gs.check()
    check(f"skew euler dim={dim} M={M} p={p} {state} {flux}", out.cpu().numpy(), D, X, mesh, um, om,
          n_exact=3 if p < 7 else 2, seed=p)


@pytest.mark.parametrize("p", [8, 10])
def test_skew_euler_high_degree_tets_sampled(p):
    """Tetrahedra p = 8 and 10 (162 curved elements, the instantiations for N = 9 and 11):
    two sampled elements against the skew oracle on their sub-mesh in FP64 and in long
    double (evaluating the oracle on the whole mesh would take minutes at these degrees)."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X = I.config_mesh(3, 3, L, p, True)
    gs = E.Skew(3, p, X, mesh.nbr_elem, mesh.nbr_face, model="euler", flux="LF")
    rng = np.random.default_rng(p)
    pick = np.sort(rng.choice(len(X), size=2, replace=False))
    D64, need, local = extended.sub_discretization(3, p, X, mesh.nbr_elem, mesh.nbr_face, pick, flux="LF",
                                                   dtype=float)
    Dx, need_x, local_x = extended.sub_discretization(3, p, X, mesh.nbr_elem, mesh.nbr_face, pick, flux="LF")
    assert np.array_equal(need, need_x) and np.array_equal(local, local_x)
    # the state: a constant admissible state (its mode 0) plus seeded N(0, 1e-3) on every mode
    # (the full-mesh projection of an analytic state would need the whole oracle mesh)
    ubar = I.conservative_from_primitive(np.array(1.2), np.array([0.3, -0.2, 0.1]), np.array(1.5))
    um = np.zeros((len(X), 5, D64.V.shape[1]))
    um[:, :, 0] = np.asarray(ubar) / D64.V[0, 0]
    um = np.ascontiguousarray(um + I.seeded_normal(200 + p, um.shape, 1e-3))
    out = gs.rhs(to_dev(um))
    torch.cuda.synchronize()
    gs.check()
    got = out.cpu().numpy()[pick]
    om = skew.EulerModel(3, dissipation=True)
    ref = skew.rhs(D64, um[need], om, "skew", local)
    rx = skew.rhs(Dx, um[need].astype(extended.EXT), om, "skew", local)
    e_gpu = np.asarray(rel_err_per_var(got, rx), dtype=float)
    e_64 = np.asarray(rel_err_per_var(ref, rx), dtype=float)
    e_flat = np.asarray(rel_err_per_var(got, ref), dtype=float)
    flat = e_64 < FLAT_REACH
    rec = dict(case=f"skew euler tet p={p} constant + noise LF (sample)", e_gpu_exact=e_gpu.tolist(),
               e_oracle64_exact=e_64.tolist(), e_gpu_oracle64=e_flat.tolist(), flat=flat.tolist(),
               n_elems=int(len(pick)), n_exact=int(len(pick)))
    _log(rec)
    print(rec)
    assert np.all(e_gpu <= C_EXACT * np.maximum(e_64, FLOOR)), ("accuracy vs exact", e_gpu, e_64)
    assert np.all(e_gpu[flat] < PARITY_TOL), ("flat bound vs exact", e_gpu, e_64)
    assert np.all(e_flat < 1e-9), ("against the FP64 oracle", e_flat)


@pytest.mark.parametrize("dim,M,p", [(2, 3, 2), (2, 4, 5), (2, 3, 9), (3, 3, 2), (3, 3, 3), (3, 3, 5)])
@pytest.mark.parametrize("upwind", [False, True])
def test_skew_advection_parity(dim, M, p, upwind):
    import torch
    mesh, X, D, um, om, gs = setup(dim, M, p, "advection", None, upwind=upwind, seed=p)
    assert gs.nc == 1
    out = gs.rhs(to_dev(um))
    torch.cuda.synchronize()
    gs.check()
    check(f"skew advection dim={dim} M={M} p={p} upwind={upwind}", out.cpu().numpy(), D, X, mesh, um, om,
          n_exact=3, seed=p)


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 3)])
def test_skew_advection_energy_on_curved_mesh(dim, p):
    """The property the skew-symmetric form was built for, on the GPU output: with the
    central interface flux the rate of the weight-adjusted energy u~^T M~ u~ / 2,
    sum_kappa u~^T M~ d u~/dt (= u^T r), vanishes to rounding on a curved periodic mesh;
    with upwinding it is negative.  M~ is recovered per element from the weight-adjusted
    inverse M~^{-1} = V^T W J^{-1} V of Eq. (weight_adjusted_inverse)."""
    import torch
    for upwind in (False, True):
        mesh, X, D, um, om, gs = setup(dim, 3, p, "advection", None, upwind=upwind, seed=7)
        dudt = gs.rhs(to_dev(um)).cpu().numpy()
        terms = []
        for e in range(D.E):
            minv = D.V.T @ ((D.ref.w / D.geo.J_vol[e])[:, None] * D.V)
            y = np.linalg.solve(minv, dudt[e, 0])          # = V^T r of element e
            terms.append(um[e, 0] * y)
        terms = np.concatenate(terms)
        rate, scale = terms.sum(), np.abs(terms).sum()
        if upwind:
            assert rate < -1e-8 * scale
        else:
            assert abs(rate) < 1e-12 * scale


def test_skew_free_stream_and_conservation_gpu():
    """Euler on curved tetrahedra: a uniform state has d u~/dt = 0 (the metric identities of
    the curl-form metrics), and sum_kappa 1^T W J V d u~/dt = 0 for a non-uniform state."""
    import torch
    from oracle import euler
    mesh, X, D, um, om, gs = setup(3, 3, 3, "euler", "density_wave")
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7, 0.2]), np.array(2.1))
    uc = np.zeros(um.shape)
    uc[:, :, 0] = ubar / D.V[0, 0]
    r = gs.rhs(to_dev(uc)).cpu().numpy()
    assert np.abs(r).max() < 1e-12 * np.abs(ubar).max()
    dudt = gs.rhs(to_dev(um)).cpu().numpy()
    cons = D.conservation_rate(dudt)
    y = np.einsum("ij,ecj->eic", D.V, dudt)
    scale = np.einsum("i,ei,eic->c", D.ref.w, D.geo.J_vol, np.abs(y))
    assert np.all(np.abs(cons) < 1e-12 * scale)
