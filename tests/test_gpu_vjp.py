"""The hand-written adjoint (esd_rhs_vjp, esd_rk_step_vjp, autograd rollout) against the
oracle's complex-step Jacobian and against central differences of the GPU forward."""
import numpy as np
import pytest

from gpu_common import workload, gpu_mesh, to_dev, check_vjp_parity, periodic_face_elements
from oracle.jacobian import jvp, rk4_jvp

pytestmark = pytest.mark.gpu

CASES = [(2, 3, 2, "vortex"), (2, 4, 4, "vortex"), (3, 3, 2, "density_wave"), (3, 3, 3, "density_wave"),
         (3, 3, 3, "tgv")]


@pytest.mark.parametrize("dim,M,p,state", CASES)
@pytest.mark.parametrize("flux", ["LF", "EC"])
def test_vjp_dot_product_against_oracle(dim, M, p, state, flux):
    """<c, J v> (oracle, complex step: exact to rounding) = <J^T c, v> (GPU adjoint)."""
    import torch
    mesh, X, D, um = workload(dim, M, p, True, flux, state)
    rng = np.random.default_rng(7)
    c = rng.standard_normal(um.shape)
    v = rng.standard_normal(um.shape)
    jv = jvp(D, um, v)
    gm = gpu_mesh(dim, p, X, mesh, flux)
    import paper_2312_07874_gb300 as E
    g = torch.empty((D.E, D.Nc, D.Np), dtype=torch.float64, device="cuda")
    E.esd_rhs_vjp(gm.handle, to_dev(um), to_dev(c), g)
    torch.cuda.synchronize()
    lhs = np.sum(c * jv)
    rhs = np.sum(g.cpu().numpy() * v)
    scale = np.sum(np.abs(c * jv))
    assert abs(lhs - rhs) < 1e-11 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("dim,M,p,state", [(2, 3, 2, "vortex"), (2, 4, 4, "vortex"), (3, 3, 2, "density_wave"),
                                         (3, 3, 3, "density_wave"), (3, 3, 3, "tgv")])
@pytest.mark.parametrize("flux", ["LF", "EC"])
def test_vjp_per_element_jacobian_transpose(dim, M, p, state, flux):
    """Per-element rows of J^T c against the oracle's complex-step Jacobian transpose in FP64
    and long double, on 6 elements (3 with a periodic facet)."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(dim, M, p, True, flux, state)
    rng = np.random.default_rng(8)
    c = rng.standard_normal(um.shape)
    gm = gpu_mesh(dim, p, X, mesh, flux)
    g = torch.empty((D.E, D.Nc, D.Np), dtype=torch.float64, device="cuda")
    E.esd_rhs_vjp(gm.handle, to_dev(um), to_dev(c), g)
    g = g.cpu().numpy()
    gm.check()
    per = periodic_face_elements(mesh)
    inner = np.setdiff1d(np.arange(D.E), per)
    sample = np.concatenate([rng.choice(per, 3, replace=False), rng.choice(inner, min(3, len(inner)), replace=False)])
    check_vjp_parity(f"vjp dim={dim} M={M} p={p} {state} {flux}", g, D, X, um, c, sample)


# Central differences of the GPU forward.  The entropy-conservative flux is smooth, so the
# plain check uses h = 1e-6.  The LF dissipation contains max(|v.n|) and max(c) over the two
# traces, which nearly coincide for a smooth state: those kinks lie within ~1e-6 of the
# state, so a difference with h = 1e-6 straddles them (error ~h, also for the oracle);
# h = 1e-7 stays on one side.  Both use Richardson extrapolation of h and 2h.
# Tetrahedra of degree 9 and 10 accumulate the per-node cotangents in global memory
# (their shared-memory footprint exceeds one CTA); the same check covers that path.
FD_CASES = [(2, 4, 3, "vortex", "EC", 1e-6), (3, 3, 3, "tgv", "EC", 1e-6),
            (2, 4, 3, "vortex", "LF", 1e-7), (3, 3, 3, "tgv", "LF", 1e-7),
            (3, 3, 8, "tgv", "EC", 1e-6), (3, 3, 9, "tgv", "EC", 1e-6), (3, 3, 10, "density_wave", "EC", 1e-6)]


@pytest.mark.parametrize("dim,M,p,state,flux,h", FD_CASES)
def test_vjp_central_differences_of_gpu_forward(dim, M, p, state, flux, h):
    """Dot-product test against central differences of esd_rhs itself (1e-6 relative)."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(dim, M, p, True, flux, state)
    gm = gpu_mesh(dim, p, X, mesh, flux)
    rng = np.random.default_rng(9)
    c = to_dev(rng.standard_normal(um.shape))
    v = to_dev(rng.standard_normal(um.shape))
    u = to_dev(um)

    def cd(hh):
        return (gm.rhs(u + hh * v) - gm.rhs(u - hh * v)) / (2 * hh)
    fd = (4.0 * cd(h) - cd(2 * h)) / 3.0
    g = torch.empty_like(u)
    E.esd_rhs_vjp(gm.handle, u, c, g)
    lhs = float((c * fd).sum())
    rhs = float((g * v).sum())
    assert abs(lhs - rhs) < 1e-6 * float((c * fd).abs().sum()), (lhs, rhs)


@pytest.mark.parametrize("dim,M,p,state", [(2, 3, 2, "vortex"), (3, 3, 2, "density_wave")])
def test_rk_step_vjp_against_oracle(dim, M, p, state):
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(dim, M, p, True, "LF", state)
    gm = gpu_mesh(dim, p, X, mesh)
    dt = 2e-3
    rng = np.random.default_rng(10)
    c = rng.standard_normal(um.shape)
    v = rng.standard_normal(um.shape)
    u = to_dev(um)
    ck = torch.empty((4,) + u.shape, dtype=torch.float64, device="cuda")
    gm.rk_step(u, dt, ck)
    cin = torch.empty_like(u)
    E.esd_rk_step_vjp(gm.handle, ck, dt, to_dev(c), cin)
    jv = rk4_jvp(D, um, v, dt)
    lhs = np.sum(c * jv)
    rhs = np.sum(cin.cpu().numpy() * v)
    assert abs(lhs - rhs) < 1e-11 * np.sum(np.abs(c * jv))
    # in place (cot_in aliases cot_out)
    cc = to_dev(c)
    E.esd_rk_step_vjp(gm.handle, ck, dt, cc, cc)
    assert torch.allclose(cc, cin, rtol=0, atol=0)


# The rollout check uses the smooth EC flux: along 80 stage evaluations the LF flux's
# max/|.| kinks are crossed even by h = 1e-7 differences; the LF step adjoint is checked
# exactly against the oracle's complex-step Jacobian in test_rk_step_vjp_against_oracle.
@pytest.mark.parametrize("checkpoint,flux,h", [("stages", "EC", 1e-6), ("steps", "EC", 1e-6)])
def test_rollout_gradient_central_differences(checkpoint, flux, h):
    """20-step RK4 rollout through torch.autograd with per-stage (or per-step) checkpoints;
    gradient of <w, u_N> against Richardson-extrapolated central differences (1e-6 relative)."""
    import torch
    from paper_2312_07874_gb300.autograd import rollout
    mesh, X, D, um = workload(3, 3, 3, True, flux, "tgv")
    gm = gpu_mesh(3, 3, X, mesh, flux)
    dt = 2e-3
    rng = np.random.default_rng(11)
    w = to_dev(rng.standard_normal(um.shape))
    v = to_dev(rng.standard_normal(um.shape))
    u0 = to_dev(um).requires_grad_(True)
    loss = (w * rollout(u0, gm, dt, 20, checkpoint)).sum()
    loss.backward()
    g = u0.grad

    def L(x):
        with torch.no_grad():
            return float((w * rollout(x, gm, dt, 20, checkpoint)).sum())

    def cd(hh):
        return (L(to_dev(um) + hh * v) - L(to_dev(um) - hh * v)) / (2 * hh)
    fd = (4.0 * cd(h) - cd(2 * h)) / 3.0
    ad = float((g * v).sum())
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


def test_vjp_torch_function():
    import torch
    from paper_2312_07874_gb300.autograd import Rhs
    mesh, X, D, um = workload(2, 3, 2, True, "LF", "vortex")
    gm = gpu_mesh(2, 2, X, mesh)
    u = to_dev(um).requires_grad_(True)
    out = Rhs.apply(u, gm)
    rng = np.random.default_rng(12)
    c = to_dev(rng.standard_normal(um.shape))
    (out * c).sum().backward()
    v = rng.standard_normal(um.shape)
    jv = jvp(D, um, v)
    assert abs(float((u.grad.cpu() * torch.from_numpy(v)).sum()) - np.sum(c.cpu().numpy() * jv)) < \
        1e-11 * np.sum(np.abs(c.cpu().numpy() * jv))


# Reverse mode with saved forward tapes: the _saved calls read the entropy-projected states
# the forward left in the tape instead of recomputing them, with the same kernels on the same
# values, so everything must agree bit for bit with the recomputing calls.
@pytest.mark.parametrize("dim,M,p,state,flux", [(2, 4, 4, "vortex", "LF"), (3, 3, 3, "tgv", "EC"),
                                               (3, 3, 4, "density_wave", "LF")])
def test_saved_tape_vjp_bitwise(dim, M, p, state, flux):
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(dim, M, p, True, flux, state)
    gm = gpu_mesh(dim, p, X, mesh, flux)
    rng = np.random.default_rng(13)
    u, c = to_dev(um), to_dev(rng.standard_normal(um.shape))
    tape = gm.empty_tapes()
    r0, r1 = torch.empty_like(u), torch.empty_like(u)
    E.esd_rhs(gm.handle, u, r0)
    E.esd_rhs_save(gm.handle, u, r1, tape)
    assert torch.equal(r0, r1)
    # the mesh workspace is overwritten by another state: the saved VJP must not read it
    E.esd_rhs(gm.handle, 1.02 * u, r0)
    g0, g1 = torch.empty_like(u), torch.empty_like(u)
    E.esd_rhs_vjp(gm.handle, u, c, g0)
    E.esd_rhs(gm.handle, 1.01 * u, r0)
    E.esd_rhs_vjp_saved(gm.handle, u, tape, c, g1)
    gm.check()
    assert torch.equal(g0, g1)
    # one RK4 step with its four stage tapes, and its adjoint
    dt = 2e-3
    ua, ub = u.clone(), u.clone()
    cka = torch.empty((4,) + u.shape, dtype=torch.float64, device="cuda")
    ckb = torch.empty_like(cka)
    tapes = gm.empty_tapes(4)
    E.esd_rk_step(gm.handle, ua, dt, cka)
    E.esd_rk_step_save(gm.handle, ub, dt, ckb, tapes)
    assert torch.equal(ua, ub) and torch.equal(cka, ckb)
    E.esd_rhs(gm.handle, 0.99 * u, r0)
    ca, cb = torch.empty_like(u), torch.empty_like(u)
    E.esd_rk_step_vjp(gm.handle, cka, dt, c, ca)
    E.esd_rk_step_vjp_saved(gm.handle, ckb, tapes, dt, c, cb)
    gm.check()
    assert torch.equal(ca, cb)


def test_saved_tape_rollout_and_rhs_function():
    """The "tapes" rollout gives the "stages" rollout's gradient bit for bit; so does the
    autograd Rhs with and without its tape."""
    import torch
    from paper_2312_07874_gb300.autograd import Rhs, rollout
    mesh, X, D, um = workload(3, 3, 3, True, "EC", "tgv")
    gm = gpu_mesh(3, 3, X, mesh, "EC")
    rng = np.random.default_rng(14)
    w = to_dev(rng.standard_normal(um.shape))
    grads = []
    for mode in ("stages", "tapes"):
        u0 = to_dev(um).requires_grad_(True)
        (w * rollout(u0, gm, 2e-3, 5, mode)).sum().backward()
        grads.append(u0.grad)
    assert torch.equal(grads[0], grads[1])
    grads = []
    for save in (False, True):
        u0 = to_dev(um).requires_grad_(True)
        (w * Rhs.apply(u0, gm, save)).sum().backward()
        grads.append(u0.grad)
    assert torch.equal(grads[0], grads[1])


def test_saved_tape_argument_checks():
    """Rejected on the host before any launch: a tape that is not 16-byte aligned, a null
    tape, and meshes without the stored pair tables."""
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(2, 3, 2, True, "LF", "vortex")
    gm = gpu_mesh(2, 2, X, mesh)
    u = to_dev(um)
    out, g = torch.empty_like(u), torch.empty_like(u)
    n = E.esd_tape_doubles(gm.handle)
    assert n % 32 == 0
    buf = torch.empty(n + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="16-byte"):
        E.esd_rhs_save(gm.handle, u, out, buf[1:])
    with pytest.raises(RuntimeError, match="16-byte"):
        E.esd_rhs_vjp_saved(gm.handle, u, buf[1:], u, g)
    otf = E.Mesh(2, 2, X, mesh.nbr_elem, mesh.nbr_face, metrics_on_the_fly=True)
    with pytest.raises(RuntimeError, match="pair tables"):
        E.esd_rhs_save(otf.handle, u, out, buf[:n])
    torch.cuda.synchronize()
