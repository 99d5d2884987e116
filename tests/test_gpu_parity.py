"""GPU parity: the CUDA path through the C ABI against the oracle, element by element.

Criteria (tests/gpu_common.py): accuracy against the oracle evaluated in long double (the
exact answer at the same FP64 inputs) within a factor 10 of the FP64 oracle's own error,
error relative to the sums of |terms| below 1e-12, and 1e-12 relative max-norm per
variable against the long-double evaluation wherever the FP64 oracle itself is within 5e-13
of it (well-conditioned variables)."""
import numpy as np
import pytest

from gpu_common import workload, gpu_mesh, to_dev, rel_err_per_var, check_parity

pytestmark = pytest.mark.gpu
TOL = 1e-12

# (dim, M, p, state): several residual tiles plus a ragged tail at each degree
RHS_CASES = [(2, 3, 1, "vortex"), (2, 5, 2, "vortex"), (2, 8, 3, "vortex"), (2, 8, 4, "vortex"),
             (2, 4, 6, "vortex"), (2, 3, 8, "vortex"), (2, 3, 10, "vortex"),
             (3, 3, 1, "density_wave"), (3, 3, 2, "density_wave"), (3, 3, 3, "density_wave"),
             (3, 3, 4, "density_wave"), (3, 3, 2, "tgv"), (3, 3, 3, "tgv"), (3, 3, 4, "tgv")]


@pytest.mark.parametrize("dim,M,p,state", RHS_CASES)
@pytest.mark.parametrize("flux", ["LF", "EC"])
def test_rhs_parity(dim, M, p, state, flux):
    """esd_rhs vs the oracle's sparse route on every element (term-scale and flat checks)
    and vs the long-double oracle on a sample (accuracy check)."""
    import torch
    mesh, X, D, um = workload(dim, M, p, True, flux, state)
    gm = gpu_mesh(dim, p, X, mesh, flux)
    u = to_dev(um)
    out = gm.rhs(u)
    torch.cuda.synchronize()
    gm.check()
    check_parity(f"rhs dim={dim} M={M} p={p} {state} {flux}", out.cpu().numpy(), D, X, um, n_exact=4, seed=p)


# Tetrahedra of degree 5..10 on the 162-element periodic mesh: the GPU computes every
# element; the FP64 oracle (slow at these degrees) a seeded sample of three elements, the
# long-double oracle one of them up to degree 7.  Degree 10 runs the facet-4 phase in two
# passes of columns.
HIGH_TET_CASES = [(5, "tgv", "LF"), (6, "tgv", "LF"), (7, "density_wave", "LF"), (8, "density_wave", "EC"),
                  (9, "tgv", "LF"), (10, "density_wave", "LF"), (10, "tgv", "EC")]


@pytest.mark.parametrize("p,state,flux", HIGH_TET_CASES)
def test_rhs_parity_high_degree_tets(p, state, flux):
    import torch
    mesh, X, D, um = workload(3, 3, p, True, flux, state)
    gm = gpu_mesh(3, p, X, mesh, flux)
    out = gm.rhs(to_dev(um)).cpu().numpy()
    gm.check()
    rng = np.random.default_rng(40 + p)
    sample = np.sort(rng.choice(D.E, size=3, replace=False))
    check_parity(f"rhs tet p={p} {state} {flux} (sample)", out[sample], D, X, um, elems=sample, n_exact=1 if p <= 7 else 0)
    # conservation over the whole GPU output (Theorem 2)
    cons = D.conservation_rate(out)
    y = np.einsum("ij,ecj->eic", D.V, out)
    scale = np.einsum("i,ei,eic->c", D.ref.w, D.geo.J_vol, np.abs(y))
    assert np.all(np.abs(cons) < 1e-11 * scale)


@pytest.mark.parametrize("dim,M,p", [(2, 5, 2), (2, 4, 5), (3, 3, 2), (3, 3, 4)])
def test_entropy_projection_parity(dim, M, p):
    import torch
    mesh, X, D, um = workload(dim, M, p)
    ref = np.transpose(D.project_entropy(um), (0, 2, 1))
    gm = gpu_mesh(dim, p, X, mesh)
    w = gm.project_entropy(to_dev(um))
    torch.cuda.synchronize()
    err = rel_err_per_var(w.cpu().numpy(), ref)
    assert np.all(err < TOL), err


@pytest.mark.parametrize("dim,M,p", [(2, 4, 3), (3, 3, 3)])
def test_l2_projection_and_nodes(dim, M, p):
    import torch
    import esd_inputs as I
    mesh, X, D, um = workload(dim, M, p)
    gm = gpu_mesh(dim, p, X, mesh)
    x = gm.volume_nodes()
    f = I.config_state_fn(dim, 2 * np.pi, "vortex" if dim == 2 else "tgv")
    un = np.transpose(f(x), (0, 2, 1))                       # [E, Nc, Nq] library node order
    got = gm.l2_project(to_dev(un))
    torch.cuda.synchronize()
    ref = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, f(D.geo.x_vol))
    err = rel_err_per_var(got.cpu().numpy(), ref)
    assert np.all(err < TOL), err


@pytest.mark.parametrize("dim,M,p", [(2, 5, 3), (3, 3, 2)])
def test_rk4_step_parity(dim, M, p):
    """One graph-captured RK4 step against the oracle's rk4_step (well-conditioned states:
    the flat 1e-12 bound on the increment u_new - u)."""
    import torch
    from oracle.timestep import rk4_step
    state = "vortex" if dim == 2 else "density_wave"
    mesh, X, D, um = workload(dim, M, p, True, "LF", state)
    dt = 1e-3
    ref = rk4_step(lambda v: D.rhs(v, "sparse"), um, dt)
    gm = gpu_mesh(dim, p, X, mesh)
    u = to_dev(um)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gm.rk_step(u, dt)           # captured into a graph on a non-default stream
        ck = torch.empty((4,) + u.shape, dtype=torch.float64, device="cuda")
        u2 = to_dev(um)
        gm.rk_step(u2, dt, ck)
    s.synchronize()
    for got in (u, u2):
        err = rel_err_per_var(got.cpu().numpy() - um, ref - um)   # compare the increments
        assert np.all(err < TOL), err
    # checkpoints hold the four stage inputs
    k1 = D.rhs(um, "sparse")
    assert np.all(rel_err_per_var(ck[0].cpu().numpy(), um) < 1e-15)
    assert np.all(rel_err_per_var(ck[1].cpu().numpy() - um, 0.5 * dt * k1) < TOL)


def test_rk4_graph_replay_matches_direct():
    import torch
    mesh, X, D, um = workload(2, 4, 3)
    gm = gpu_mesh(2, 3, X, mesh)
    a, b = to_dev(um), to_dev(um)
    s = torch.cuda.Stream()
    for _ in range(3):
        with torch.cuda.stream(s):
            gm.rk_step(a, 2e-3)
        import paper_2312_07874_gb300 as E
        E.lib().esd_rk_step(gm.handle, E._ptr(b), 2e-3, None, None)   # legacy stream: direct launches
        torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("dim,M,p", [(2, 4, 3), (3, 3, 3)])
def test_diagnostics_theorems(dim, M, p):
    """Theorem 2 (conservation) and Theorem 4 (entropy conservation with EC facets) on the GPU."""
    import torch
    mesh, X, D, um = workload(dim, M, p, True, "EC")
    gm = gpu_mesh(dim, p, X, mesh, "EC")
    u = to_dev(um)
    d = gm.diagnostics(u).cpu().numpy()
    dudt = gm.rhs(u).cpu().numpy()
    nc = dim + 2
    scale = np.abs(d[nc + 1])
    assert abs(d[nc]) < 1e-12 * scale
    # the oracle's own statement of both theorems evaluated on the GPU's du/dt
    ent, ent_scale = D.entropy_rate(um, dudt)
    assert abs(ent) < 1e-12 * ent_scale
    cons = D.conservation_rate(dudt)
    y = np.einsum("ij,ecj->eic", D.V, dudt)
    cscale = np.einsum("i,ei,eic->c", D.ref.w, D.geo.J_vol, np.abs(y))
    # the per-element sums are differences of facet fluxes, which carry the low-Mach
    # pressure (~71) and exceed |d u~/dt| here by ~10-100x; 1e-12 of this scale is the bound
    assert np.all(np.abs(cons) < 1e-12 * cscale)
    assert np.all(np.abs(d[:nc]) < 1e-11 * cscale)


@pytest.mark.parametrize("dim,p", [(2, 4), (3, 3)])
def test_free_stream_gpu(dim, p):
    import torch
    from oracle import euler
    mesh, X, D, _ = workload(dim, 3, p)
    ubar = euler.conservative(np.array(1.3), np.array([0.4, -0.7, 0.2][:dim]), np.array(2.1))
    um = np.einsum("ij,i,eic->ecj", D.V, D.ref.w, np.broadcast_to(ubar, (D.E, D.ref.Nq, D.Nc)))
    gm = gpu_mesh(dim, p, X, mesh)
    out = gm.rhs(to_dev(um)).cpu().numpy()
    assert np.abs(out).max() < 1e-12 * np.abs(ubar).max()


def test_invalid_arguments_rejected_before_launch():
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(2, 3, 2)
    gm = gpu_mesh(2, 2, X, mesh)
    u = to_dev(um)
    host = np.zeros(um.shape)
    st = E.lib().esd_rhs(gm.handle, E.ctypes.c_void_p(host.ctypes.data), E._ptr(u), None)
    assert st == -1
    st = E.lib().esd_rhs(gm.handle, E._ptr(u), E._ptr(u), None)   # aliasing
    assert st == -1
    st = E.lib().esd_rk_step(gm.handle, E._ptr(u), -1.0, None, None)
    assert st == -1


def test_non_admissible_state_flagged():
    """A negative density in the input is reported as ESD_ERR_STATE by esd_mesh_check
    (host-side detection of a device flag; nothing faults)."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(2, 3, 2)
    gm = gpu_mesh(2, 2, X, mesh)
    bad = um.copy()
    bad[3, 0, 0] = -abs(bad[3, 0, 0]) * 3
    gm.rhs(to_dev(bad))
    with pytest.raises(E.EsdError) as ex:
        gm.check()
    assert ex.value.status == -4
    gm.rhs(to_dev(um))
    gm.check()


def test_affine_triangles_rhs_and_ten_rk4_steps():
    """The plain-method triangle workload exactly: [0, 2 pi]^2 periodic, 8 x 8 x 2 = 128 affine
    triangles, p = 2, isentropic vortex (strength 5 at the centre, background rho = u = v =
    p = 1), LF interface flux.  One esd_rhs against the oracle, then 10 RK4 steps at CFL 0.1
    (dt = CFL h / (lambda_max (2p + 1)), h = L/M), captured once in a CUDA graph and
    replayed, against 10 steps of the oracle's RK4 (flat 1e-12 on the total change)."""
    import torch
    import esd_inputs as I
    from oracle.timestep import rk4_step
    dim, M, p, L = 2, 8, 2, 2 * np.pi
    mesh, X, D, um = workload(dim, M, p, False, "LF", "vortex", 0.0)
    gm = gpu_mesh(dim, p, X, mesh)
    u = to_dev(um)
    out = gm.rhs(u)
    torch.cuda.synchronize()
    gm.check()
    check_parity("affine triangles p=2 vortex rhs", out.cpu().numpy(), D, X, um, n_exact=4, seed=1)
    lam = I.max_wave_speed_sampled(I.config_state_fn(dim, L, "vortex"), dim, L)
    dt = 0.1 * (L / M) / (lam * (2 * p + 1))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(10):
            gm.rk_step(u, dt)       # first call captures the graph, the others replay it
    s.synchronize()
    gm.check()
    ref = um
    for _ in range(10):
        ref = rk4_step(lambda v: D.rhs(v, "sparse"), ref, dt)
    err = rel_err_per_var(u.cpu().numpy() - um, ref - um)
    assert np.all(err < TOL), err


OTF_CASES = [(2, 4, 3, "vortex"), (2, 3, 8, "vortex"), (3, 3, 2, "tgv"), (3, 3, 4, "density_wave"),
             (3, 3, 4, "tgv"), (3, 3, 7, "density_wave")]


@pytest.mark.parametrize("dim,M,p,state", OTF_CASES)
def test_metrics_on_the_fly_parity(dim, M, p, state):
    """A mesh created with ESD_MESH_METRICS_ON_THE_FLY forms every pair direction from the
    per-node metric terms in the kernel: the same checks against the oracle as the stored
    tables, the same result as the stored-table mesh up to rounding, and an RK4 step; the
    VJP and batches report ESD_ERR_UNSUPPORTED."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(dim, M, p, True, "LF", state)
    g_otf = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux="LF", metrics_on_the_fly=True)
    g_tab = gpu_mesh(dim, p, X, mesh)
    u = to_dev(um)
    a = g_otf.rhs(u).cpu().numpy()
    b = g_tab.rhs(u).cpu().numpy()
    g_otf.check()
    if p <= 4:
        check_parity(f"on-the-fly directions dim={dim} M={M} p={p} {state}", a, D, X, um, n_exact=2, seed=p)
    else:
        rng = np.random.default_rng(p)
        sample = np.sort(rng.choice(D.E, size=3, replace=False))
        check_parity(f"on-the-fly directions dim={dim} M={M} p={p} {state} (sample)", a[sample], D, X, um,
                     elems=sample, n_exact=1, seed=p)
    # against the stored-table mesh: relative to the term scale the two differ by rounding only
    assert np.all(rel_err_per_var(a, b) < 1e-9)
    assert g_otf.info["device_bytes"] < g_tab.info["device_bytes"]
    ua, ub = u.clone(), u.clone()
    g_otf.rk_step(ua, 1e-3)
    g_tab.rk_step(ub, 1e-3)
    torch.cuda.synchronize()
    assert np.all(rel_err_per_var(ua.cpu().numpy() - um, ub.cpu().numpy() - um) < 1e-9)
    g = torch.empty_like(u)
    assert E.lib().esd_rhs_vjp(g_otf.handle, E._ptr(u), E._ptr(u), E._ptr(g), None) == -7
    with pytest.raises(E.EsdError) as ex:
        E.esd_batch_create([g_otf.handle])
    assert ex.value.status == -7
