"""Element partitions on one GPU: a mesh split into partition meshes (local elements plus
ghosts) evaluated phase by phase with an explicit facet-trace exchange between them
(esd_rhs_begin -> esd_part_export / esd_part_import -> esd_rhs_end, and the VJP with its
cotangent exchange) must reproduce the unsplit mesh's right-hand side and VJP bit for bit,
since every element runs the same per-element arithmetic on the same inputs."""
import numpy as np
import pytest

from gpu_common import workload, gpu_mesh, to_dev

pytestmark = pytest.mark.gpu


def _owners(X, kind, P):
    E = X.shape[0]
    if kind == "round_robin":
        return np.arange(E) % P
    c = X.mean(axis=1)[:, 0]
    edges = np.quantile(c, np.linspace(0, 1, P + 1)[1:-1])
    return np.searchsorted(edges, c, side="right")


def _parts(dim, p, X, mesh, flux, kind, P):
    import paper_2312_07874_gb300 as E
    from paper_2312_07874_gb300.partition import split
    parts = split(mesh.nbr_elem, mesh.nbr_face, _owners(X, kind, P))
    meshes = [E.Mesh(dim, p, pt.map_nodes(X), pt.nbr_elem, pt.nbr_face, flux=flux, n_ghost=pt.n_ghost)
              for pt in parts]
    return parts, meshes


@pytest.mark.parametrize("dim,M,p,state,flux,kind,P", [
    (2, 4, 4, "vortex", "LF", "slab", 2),
    (2, 4, 3, "vortex", "EC", "round_robin", 3),
    (3, 3, 3, "tgv", "LF", "slab", 2),
    (3, 3, 4, "density_wave", "EC", "round_robin", 3),
    (3, 3, 7, "tgv", "LF", "round_robin", 2),   # two lanes per line task (tetrahedra p >= 7)
])
def test_split_mesh_matches_unsplit(dim, M, p, state, flux, kind, P):
    import torch
    import paper_2312_07874_gb300 as E
    from paper_2312_07874_gb300.partition import exchange_local
    mesh, X, D, um = workload(dim, M, p, True, flux, state)
    gm = gpu_mesh(dim, p, X, mesh, flux)
    rng = np.random.default_rng(21)
    u, c = to_dev(um), to_dev(rng.standard_normal(um.shape))
    ref, gref = torch.empty_like(u), torch.empty_like(u)
    E.esd_rhs(gm.handle, u, ref)
    E.esd_rhs_vjp(gm.handle, u, c, gref)
    parts, meshes = _parts(dim, p, X, mesh, flux, kind, P)
    assert all(pt.n_ghost > 0 for pt in parts)
    loc = [torch.from_numpy(pt.local).to("cuda") for pt in parts]
    ul = [u[i].contiguous() for i in loc]
    cl = [c[i].contiguous() for i in loc]
    # d u~/dt: projection, trace exchange, residual
    out = [torch.empty_like(x) for x in ul]
    for m, x in zip(meshes, ul):
        E.esd_rhs_begin(m.handle, x)
    exchange_local(meshes, parts, E.ESD_TRACE_STATES)
    for m, o in zip(meshes, out):
        E.esd_rhs_end(m.handle, o)
    for m in meshes:
        m.check()
    for i, o in zip(loc, out):
        assert torch.equal(o, ref[i])
    # VJP: projection, trace exchange, residual adjoint, cotangent exchange, projection adjoint
    grad = [torch.empty_like(x) for x in ul]
    for m, x in zip(meshes, ul):
        E.esd_rhs_begin(m.handle, x)
    exchange_local(meshes, parts, E.ESD_TRACE_STATES)
    for m, cc in zip(meshes, cl):
        E.esd_rhs_vjp_mid(m.handle, cc)
    exchange_local(meshes, parts, E.ESD_TRACE_COTANGENTS)
    for m, x, g in zip(meshes, ul, grad):
        E.esd_rhs_vjp_end(m.handle, x, g)
    for m in meshes:
        m.check()
    for i, g in zip(loc, grad):
        assert torch.equal(g, gref[i])


def test_phases_on_an_ordinary_mesh():
    """Without ghosts the phases compose to esd_rhs and esd_rhs_vjp."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(3, 3, 2, True, "LF", "tgv")
    gm = gpu_mesh(3, 2, X, mesh)
    rng = np.random.default_rng(22)
    u, c = to_dev(um), to_dev(rng.standard_normal(um.shape))
    a, b, ga, gb = (torch.empty_like(u) for _ in range(4))
    E.esd_rhs(gm.handle, u, a)
    E.esd_rhs_begin(gm.handle, u)
    E.esd_rhs_end(gm.handle, b)
    E.esd_rhs_vjp(gm.handle, u, c, ga)
    E.esd_rhs_begin(gm.handle, u)
    E.esd_rhs_vjp_mid(gm.handle, c)
    E.esd_rhs_vjp_end(gm.handle, u, gb)
    gm.check()
    assert torch.equal(a, b) and torch.equal(ga, gb)


def test_partition_argument_checks():
    """Whole-RHS calls are refused on partition meshes; ghost ranges and trace kinds are
    checked on the host; an export index outside the partition sends zeros and is reported
    by esd_mesh_check (the kernel checks every index before reading)."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(2, 4, 2, True, "LF", "vortex")
    parts, meshes = _parts(2, 2, X, mesh, "LF", "slab", 2)
    m, pt = meshes[0], parts[0]
    u = to_dev(um)[torch.from_numpy(pt.local).to("cuda")].contiguous()
    out = torch.empty_like(u)
    for call in (lambda: E.esd_rhs(m.handle, u, out), lambda: m.rk_step(u.clone(), 1e-3),
                 lambda: E.esd_rhs_vjp(m.handle, u, u, out)):
        with pytest.raises(RuntimeError, match="partition"):
            call()
    ng, per_s, per_c = E.esd_part_info(m.handle)
    assert ng == pt.n_ghost and per_s == 8 * 9 and per_c == 4 * 9   # (dim + 6) N_f N_fq, (dim + 2) N_f N_fq
    buf = torch.zeros((ng + 1, per_s), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="ghost range"):
        E.esd_part_import(m.handle, E.ESD_TRACE_STATES, buf, 0, ng + 1)
    with pytest.raises(RuntimeError, match="ghost range"):
        E.esd_part_import(m.handle, E.ESD_TRACE_STATES, buf, -1, 1)
    with pytest.raises(RuntimeError, match="kind"):
        E.esd_part_import(m.handle, 7, buf, 0, 1)
    E.esd_rhs_begin(m.handle, u)
    bad = torch.tensor([0, pt.n_local, -1], dtype=torch.int64, device="cuda")
    msg = torch.full((3, per_s), 5.0, dtype=torch.float64, device="cuda")
    E.esd_part_export(m.handle, E.ESD_TRACE_STATES, bad, msg)
    with pytest.raises(RuntimeError, match="outside"):
        m.check()
    assert torch.all(msg[1:] == 0) and torch.all(torch.isfinite(msg[0]))
    assert float(msg[0, 0]) > 0 and float(msg[0, 3 * 9]) > 0   # rho and p at the first facet node
    m.check()   # the flag was cleared by the report
