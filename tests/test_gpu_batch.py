"""Batched persistent execution of many meshes (esd_batch_*): against the oracle (sampled
elements of every mesh of a mixed batch; whole small meshes for the RK4 step) and against
the plain per-mesh path (bitwise)."""
import numpy as np
import pytest

from gpu_common import check_parity, rel_err_per_var

pytestmark = pytest.mark.gpu

MIX = [(2, 3, 2, "vortex"), (2, 4, 4, "vortex"), (3, 3, 2, "tgv"), (2, 3, 7, "vortex"), (3, 3, 3, "density_wave"),
       (3, 4, 1, "tgv"), (3, 3, 9, "tgv"), (3, 3, 3, "tgv")]


def _meshes(with_arrays=False):
    import torch
    import esd_inputs as I
    import paper_2312_07874_gb300 as E
    out = []
    for k, (dim, M, p, state) in enumerate(MIX):
        L = 2 * np.pi
        mesh, X = I.config_mesh(dim, M, L, p, True)
        gm = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face)
        x = gm.volume_nodes()
        un = np.ascontiguousarray(np.transpose(I.config_state_fn(dim, L, state)(x), (0, 2, 1)))
        u = gm.l2_project(torch.from_numpy(un).cuda())
        u += 1e-3 * torch.from_numpy(I.seeded_normal(30 + k, tuple(u.shape), 1.0)).cuda()
        out.append((gm, u, mesh, X) if with_arrays else (gm, u))
    return out


def test_batch_rhs_against_oracle():
    """One esd_batch_rhs over the mixed batch (triangles and tetrahedra, p = 1..9, element
    counts that leave ragged last tiles): every mesh's output on sampled elements (its last
    element included) against the oracle, FP64 and, up to p = 7, long double."""
    import torch
    import paper_2312_07874_gb300 as E
    from oracle import extended
    ms = _meshes(with_arrays=True)
    b = E.esd_batch_create([m.handle for m, *_ in ms])
    outs = [torch.empty_like(u) for _, u, *_ in ms]
    E.esd_batch_rhs(b, [u for _, u, *_ in ms], outs)
    torch.cuda.synchronize()
    for k, ((gm, u, mesh, X), o) in enumerate(zip(ms, outs)):
        gm.check()
        dim, M, p, state = MIX[k]
        rng = np.random.default_rng(60 + k)
        sample = np.unique(np.append(rng.choice(mesh.n_elem, 3, replace=False), mesh.n_elem - 1))
        Ds, need, local = extended.sub_discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face, sample,
                                                      dtype=np.float64)
        um = u.cpu().numpy()[need]
        check_parity(f"batch rhs mesh {k}: dim={dim} M={M} p={p} {state}", o.cpu().numpy()[sample], Ds,
                     X[need], um, elems=local, n_exact=1 if p <= 7 else 0, seed=k)
    E.esd_batch_destroy(b)


def test_batch_rk_step_against_oracle():
    """One esd_batch_rk_step over a mixed batch of whole small meshes against the oracle's
    RK4 step of each mesh (increments, 1e-12 relative per variable: well-conditioned states)."""
    import torch
    import esd_inputs as I
    import paper_2312_07874_gb300 as E
    from oracle.residual import Discretization
    from oracle.timestep import rk4_step
    mix = [(2, 3, 2, "vortex"), (3, 3, 1, "density_wave"), (2, 4, 3, "vortex"), (3, 3, 2, "density_wave")]
    L = 2 * np.pi
    Ds, gms, us, ums, dts = [], [], [], [], []
    for k, (dim, M, p, state) in enumerate(mix):
        mesh, X = I.config_mesh(dim, M, L, p, True)
        D = Discretization(dim, p, X, mesh.nbr_elem, mesh.nbr_face)
        um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, I.config_state_fn(dim, L, state)(D.geo.x_vol))
        um = np.ascontiguousarray(um + I.seeded_normal(70 + k, um.shape, 1e-3))
        Ds.append(D)
        gms.append(E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face))
        ums.append(um)
        us.append(torch.from_numpy(um).cuda())
        dts.append(2e-3 * (1 + 0.25 * k))
    b = E.esd_batch_create([m.handle for m in gms])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        E.esd_batch_rk_step(b, us, dts)
    s.synchronize()
    for D, gm, u, um, dt in zip(Ds, gms, us, ums, dts):
        gm.check()
        ref = rk4_step(lambda v: D.rhs(v, "sparse"), um, dt)
        err = rel_err_per_var(u.cpu().numpy() - um, ref - um)
        assert np.all(err < 1e-12), err
    E.esd_batch_destroy(b)


def test_batch_rhs_equals_per_mesh():
    import torch
    import paper_2312_07874_gb300 as E
    ms = _meshes()
    b = E.esd_batch_create([m.handle for m, _ in ms])
    outs = [torch.empty_like(u) for _, u in ms]
    for _ in range(2):   # second call replays the captured graph
        E.esd_batch_rhs(b, [u for _, u in ms], outs)
        torch.cuda.synchronize()
    for (m, u), o in zip(ms, outs):
        ref = m.rhs(u)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)
    E.esd_batch_destroy(b)


def test_batch_rk_step_equals_per_mesh():
    import torch
    import paper_2312_07874_gb300 as E
    ms = _meshes()
    ua = [u.clone() for _, u in ms]
    ub = [u.clone() for _, u in ms]
    # a stable step for each mesh: CFL 0.1 (h / (lambda (2p+1))), varied per mesh
    dts = [0.1 * (2 * np.pi / M) / (12.0 * (2 * p + 1)) * (1 + 0.1 * k)
           for k, (_, M, p, _) in enumerate(MIX)]
    b = E.esd_batch_create([m.handle for m, _ in ms])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            E.esd_batch_rk_step(b, ua, dts)
            for (m, _), u, dt in zip(ms, ub, dts):
                m.rk_step(u, dt)
    s.synchronize()
    for a, c in zip(ua, ub):
        assert torch.equal(a, c)
    E.esd_batch_destroy(b)


@pytest.mark.parametrize("waves", [0, 1, 1000])
def test_batch_with_meshes_on_their_own_launches(waves):
    """Large members of a batch run their own launches inside the batch graph (waves = 0:
    every mesh; waves = 1, the default: the meshes whose residual launch fills a wave, next
    to the persistent launches of the others; 1000: every mesh in the persistent launches):
    d u~/dt and the RK4 step stay bitwise equal to the per-mesh path."""
    import torch
    import paper_2312_07874_gb300 as E
    ms = _meshes()
    E.lib().esd_debug_batch_solo_waves(waves)
    try:
        b = E.esd_batch_create([m.handle for m, _ in ms])
    finally:
        E.lib().esd_debug_batch_solo_waves(1)
    outs = [torch.empty_like(u) for _, u in ms]
    E.esd_batch_rhs(b, [u for _, u in ms], outs)
    torch.cuda.synchronize()
    for (m, u), o in zip(ms, outs):
        assert torch.equal(o, m.rhs(u))
    ua = [u.clone() for _, u in ms]
    ub = [u.clone() for _, u in ms]
    dts = [0.1 * (2 * np.pi / M) / (12.0 * (2 * p + 1)) for (_, M, p, _) in MIX]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            E.esd_batch_rk_step(b, ua, dts)
            for (m, _), u, dt in zip(ms, ub, dts):
                m.rk_step(u, dt)
    s.synchronize()
    for a, c in zip(ua, ub):
        assert torch.equal(a, c)
    E.esd_batch_destroy(b)
    assert E.lib().esd_debug_batch_solo_waves(-1) != 0


def test_autotune_subset_and_invalid_bits():
    import torch
    import paper_2312_07874_gb300 as E
    ms = _meshes()
    m, u = ms[4]
    before = m.rhs(u)
    info0 = dict(m.info)
    m.autotune(u, E.ESD_TUNE_ADJOINT)        # the forward shapes stay as they were
    assert m.info["elems_per_cta_residual"] == info0["elems_per_cta_residual"]
    assert m.info["elems_per_cta_project"] == info0["elems_per_cta_project"]
    with pytest.raises(E.EsdError) as ex:
        m.autotune(u, 8)
    assert ex.value.status == -1
    after = m.rhs(u)
    torch.cuda.synchronize()
    assert torch.equal(before, after)


def test_autotune_keeps_results_and_valid_shapes():
    import torch
    import paper_2312_07874_gb300 as E
    ms = _meshes()
    for m, u in ms[:3]:
        before = m.rhs(u)
        info = m.autotune(u)
        assert info["elems_per_cta_project"] >= 1 and info["elems_per_cta_residual"] >= 1
        after = m.rhs(u)
        torch.cuda.synchronize()
        assert torch.equal(before, after)


def test_graph_caches_evict_and_recapture():
    """More argument sets than the 16 cached graphs: every call still gives the per-mesh
    result, including a set whose graph was dropped and is captured again."""
    import torch
    import paper_2312_07874_gb300 as E
    ms = _meshes()[:3]
    b = E.esd_batch_create([m.handle for m, _ in ms])
    refs = [m.rhs(u) for m, u in ms]
    first = None
    for k in range(18):
        outs = [torch.empty_like(u) for _, u in ms]
        E.esd_batch_rhs(b, [u for _, u in ms], outs)
        torch.cuda.synchronize()
        assert all(torch.equal(o, r) for o, r in zip(outs, refs))
        first = first or outs
    for o in first:
        o.zero_()
    E.esd_batch_rhs(b, [u for _, u in ms], first)
    torch.cuda.synchronize()
    assert all(torch.equal(o, r) for o, r in zip(first, refs))
    E.esd_batch_destroy(b)
    # per-mesh RK4 graphs: 18 step sizes on a side stream against direct launches on the
    # legacy stream (no graph)
    m, u0 = ms[0]
    s = torch.cuda.Stream()
    for k in range(18):
        dt = 1e-3 * (1 + 0.05 * k)
        a, c = u0.clone(), u0.clone()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            m.rk_step(a, dt)
        s.synchronize()
        m.rk_step(c, dt)
        torch.cuda.synchronize()
        assert torch.equal(a, c)
