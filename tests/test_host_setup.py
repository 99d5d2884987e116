"""CPU checks of the CUDA library's host setup (C++, independent of the oracle) against
the oracle: quadrature/metric data, pair coefficients of the line-based flux
differencing, and facet connectivity.  No GPU is touched (esd_debug_host_setup)."""
import ctypes
import os
import re
from functools import lru_cache

import numpy as np
import pytest

import esd_inputs as I
from oracle.reference import RefElement
from oracle.geometry import Geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2312_07874_gb300", "libesd.so")
pytestmark = pytest.mark.skipif(not os.path.exists(LIB), reason="libesd.so not built")


def test_library_exports_every_declared_symbol():
    inc = os.path.join(ROOT, "include")
    header = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    names = set(re.findall(r"\b(esd_[a-z0-9_]+)\s*\(", header))
    lib = ctypes.CDLL(LIB)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert len(names) >= 20


@lru_cache(maxsize=None)
def both(dim, M, p, warp):
    import paper_2312_07874_gb300 as E
    L = 2 * np.pi
    mesh, X = I.config_mesh(dim, M, L, p, warp)
    out, info = E.esd_debug_host_setup(dim, p, X, mesh.nbr_elem, mesh.nbr_face)
    ref = RefElement(dim, p)
    geo = Geometry(ref, X, mesh.nbr_elem, mesh.nbr_face)
    return mesh, out, info, ref, geo


@lru_cache(maxsize=None)
def ulp_geometry(dim, M, p, warp):
    """The oracle's geometry after a one-ulp relative perturbation of every mapping node:
    its change is the rounding sensitivity of the metric data, which grows with the degree
    of the equispaced-lattice interpolant (its derivatives amplify node errors)."""
    mesh, X = I.config_mesh(dim, M, 2 * np.pi, p, warp)
    rng = np.random.default_rng(3)
    Xp = X * (1.0 + np.finfo(float).eps * rng.choice([-1.0, 1.0], size=X.shape))
    return Geometry(RefElement(dim, p), Xp, mesh.nbr_elem, mesh.nbr_face)


def vol_map(dim, n):
    """oracle index (alpha_1 slowest) of each library volume node (c_1 fastest)."""
    idx = []
    for v in range(n ** dim):
        c = [v % n, (v // n) % n, v // (n * n)][:dim]
        o = 0
        for k in range(dim):
            o = o * n + c[k]
        idx.append(o)
    return np.array(idx)


def fac_map(dim, n):
    if dim == 2:
        return np.arange(n)
    return np.array([(j % n) * n + j // n for j in range(n * n)])


CASES = [(2, 3, 1, True), (2, 3, 3, True), (2, 3, 4, False), (3, 3, 1, True), (3, 3, 2, True), (3, 3, 4, True),
         (3, 3, 7, True), (3, 3, 10, True)]


@pytest.mark.parametrize("dim,M,p,warp", CASES)
def test_geometry_matches_oracle(dim, M, p, warp):
    mesh, out, info, ref, geo = both(dim, M, p, warp)
    n = p + 1
    vm = vol_map(dim, n)
    fm = fac_map(dim, n)
    assert np.allclose(out["xvol"], geo.x_vol[:, vm], rtol=0, atol=1e-13)
    wj = ref.w[vm][None] * geo.J_vol[:, vm]
    assert np.abs(out["wj"] - wj).max() < 1e-13 * np.abs(wj).max()
    Nqf = ref.Nqf
    # bound: 1e-12 absolute for unit normals (1e-13 relative for B J), or 20 x the oracle's
    # own one-ulp sensitivity where that is larger (high degrees)
    gp = ulp_geometry(dim, M, p, warp)
    for z in range(ref.Nf):
        bj = ref.wf[z][fm][None] * geo.Jf[z][:, fm]
        kb = np.abs(geo.Jf[z] - gp.Jf[z]).max() / np.abs(geo.Jf[z]).max()
        assert np.abs(out["bj"][:, z * Nqf:(z + 1) * Nqf] - bj).max() < max(1e-13, 20 * kb) * np.abs(bj).max()
        kn = np.abs(geo.n_fac[z] - gp.n_fac[z]).max()
        for m in range(dim):
            err = np.abs(out["nrm"][:, m, z * Nqf:(z + 1) * Nqf] - geo.n_fac[z][:, fm, m]).max()
            assert err < max(1e-12, 20 * kn), (err, kn)


def pair_slots(dim, n):
    """(phase offset, slot, task, volume node, partner) for every library pair, mirroring
    the task structure of the residual kernel; partner is ('v', node) or ('f', facet node)."""
    T = n ** (dim - 1)
    Lv = n * (n - 1) // 2
    Nqf = n ** (dim - 1)
    vol, fac = [], []
    for ph in range(dim):
        for t in range(T):
            m = 0
            for a in range(n):
                for b in range(a + 1, n):
                    if dim == 2:
                        vi, vj = (a + n * t, b + n * t) if ph == 0 else (t + n * a, t + n * b)
                    else:
                        t0, t1 = t % n, t // n
                        if ph == 0:
                            vi, vj = a + n * t, b + n * t
                        elif ph == 1:
                            vi, vj = t0 + n * (a + n * t1), t0 + n * (b + n * t1)
                        else:
                            vi, vj = t + n * n * a, t + n * n * b
                    vol.append((ph * Lv + m, t, vi, vj))
                    m += 1
    off0 = 0
    off1 = 2 * n * dim * T
    for t in range(T):
        for a in range(n):
            fac.append((off0, a, t, a + n * t, 1 * Nqf + t))
            fac.append((off0, n + a, t, a + n * t, 2 * Nqf + t))
        for b in range(n):
            vi = t + n * b if dim == 2 else (t % n) + n * (b + n * (t // n))
            fac.append((off1, b, t, vi, t))
        if dim == 3:
            off3 = off1 + n * dim * T
            a, b2 = t % n, t // n
            m = 0
            for bp in range(n):
                for b3 in range(n):
                    fac.append((off3, m, t, a + n * (b2 + n * b3), 3 * Nqf + a + n * bp))
                    m += 1
    return vol, fac, T


@pytest.mark.parametrize("dim,M,p,warp", CASES)
def test_pair_coefficients_match_assembled_operators(dim, M, p, warp):
    """Library line-pair directions equal sum_l S^(l)_ij (G_l.(i) + G_l.(j)) from the oracle's
    assembled S^(l), and facet-pair directions equal [R^T B]_ij {{J n}}_ij (Section 5.1);
    the library stores both halved."""
    mesh, out, info, ref, geo = both(dim, M, p, warp)
    n = p + 1
    vm = vol_map(dim, n)
    fm = fac_map(dim, n)
    vol, fac, T = pair_slots(dim, n)
    assert len(vol) == info["vol_pairs_per_elem"] and len(fac) == info["facet_pairs_per_elem"]
    E = geo.E
    gp = ulp_geometry(dim, M, p, warp)
    # 2e-13 relative, or 20 x the oracle's one-ulp sensitivity of the metric terms
    tol = max(2e-13, 20 * np.abs(gp.G_vol - geo.G_vol).max() / np.abs(geo.G_vol).max(),
              20 * max(np.abs(a - b).max() / np.abs(a).max() for a, b in zip(geo.Jn_fac, gp.Jn_fac)))
    vdir = out["vdir"].reshape(E, -1)
    scale = np.abs(vdir).max()
    for slot, t, vi, vj in vol:
        i, j = vm[vi], vm[vj]
        expect = sum(ref.S[l][i, j] * (geo.G_vol[:, i, l, :] + geo.G_vol[:, j, l, :]) for l in range(dim))
        got = 2.0 * np.stack([vdir[:, (slot * dim + k) * T + t] for k in range(dim)], -1)   # stored halved
        assert np.abs(got - expect).max() < tol * scale
    # every structurally nonzero S entry is covered exactly once
    covered = {(vm[vi], vm[vj]) for _, _, vi, vj in vol}
    nz = set()
    for l in range(dim):
        I_, J_ = np.nonzero(np.triu(ref.S[l], 1))
        nz |= set(zip(I_.tolist(), J_.tolist()))
    assert covered == nz
    fdir = out["fdir"].reshape(E, -1)
    fscale = np.abs(fdir).max()
    Nqf = ref.Nqf
    seen = set()
    for off, slot, t, vi, f in fac:
        z, j = f // Nqf, fm[f % Nqf]
        i = vm[vi]
        RB = (ref.R[z].T @ ref.B[z])[i, j]
        JnV = np.einsum("elm,l->em", geo.G_vol[:, i], ref.nhat[z])
        expect = RB * 0.5 * (JnV + geo.Jn_fac[z][:, j])
        got = 2.0 * np.stack([fdir[:, off + (slot * dim + k) * T + t] for k in range(dim)], -1)
        assert np.abs(got - expect).max() < tol * fscale
        seen.add((z, i, j))
    nnz = sum(np.count_nonzero(R.T @ B) for R, B in zip(ref.R, ref.B))
    assert len(seen) == nnz == info["facet_pairs_per_elem"]


@pytest.mark.parametrize("dim,M,p,warp", CASES)
def test_facet_connectivity_matches_oracle(dim, M, p, warp):
    mesh, out, info, ref, geo = both(dim, M, p, warp)
    n = p + 1
    fm = fac_map(dim, n)
    inv = np.argsort(fm)
    Nqf = ref.Nqf
    for e in range(geo.E):
        for z in range(ref.Nf):
            for jl in range(Nqf):
                f = z * Nqf + jl
                e2, f2 = out["nbr"][e, f], out["nbr_node"][e, f]
                assert e2 == mesh.nbr_elem[e, z] and f2 // Nqf == mesh.nbr_face[e, z]
                assert fm[f2 % Nqf] == geo.perm[e, z, fm[jl]]


def test_invalid_meshes_rejected():
    import paper_2312_07874_gb300 as E
    mesh, X = I.config_mesh(3, 3, 2 * np.pi, 2, True)
    bad = X.copy()
    bad[5] = bad[5][:, [1, 0, 2]]            # reflect one element: J < 0
    with pytest.raises(E.EsdError) as ex:
        E.esd_debug_host_setup(3, 2, bad, mesh.nbr_elem, mesh.nbr_face)
    assert ex.value.status == -2
    nb = mesh.nbr_elem.copy()
    nb[0, 0] = (nb[0, 0] + 1) % mesh.n_elem     # asymmetric connectivity
    with pytest.raises(E.EsdError) as ex:
        E.esd_debug_host_setup(3, 2, X, nb, mesh.nbr_face)
    assert ex.value.status == -2
    with pytest.raises(E.EsdError) as ex:
        E.esd_debug_host_setup(3, 11, I.config_mesh(3, 3, 1.0, 1, False)[1], mesh.nbr_elem, mesh.nbr_face)
    assert ex.value.status in (-1, -7)


def test_empty_mesh_rejected():
    import paper_2312_07874_gb300 as E
    with pytest.raises(E.EsdError) as ex:
        E.esd_debug_host_setup(3, 2, np.zeros((0, 10, 3)), np.zeros((0, 4), np.int32), np.zeros((0, 4), np.int8))
    assert ex.value.status == -1
    with pytest.raises(E.EsdError) as ex:
        E.esd_debug_host_setup(2, 2, np.zeros((0, 6, 2)), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int8))
    assert ex.value.status == -1


def test_kernel_layouts_audited_for_every_degree():
    """Shared-memory layouts, bulk-copy sizes and default launch shapes of every supported
    (dim, p), checked on the host before any kernel runs (esd_debug_check_layouts)."""
    import paper_2312_07874_gb300 as E
    E.esd_debug_check_layouts()
