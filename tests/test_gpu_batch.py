"""Batched persistent execution of many meshes (esd_batch_*) against the plain per-mesh path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MIX = [(2, 3, 2, "vortex"), (2, 4, 4, "vortex"), (3, 3, 2, "tgv"), (2, 3, 7, "vortex"), (3, 3, 3, "density_wave"),
       (3, 4, 1, "tgv"), (3, 3, 9, "tgv"), (3, 3, 3, "tgv")]


def _meshes():
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
        out.append((gm, u))
    return out


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
