"""esd_rhs_static_scratch: the esd_rhs variant for callers that cannot allocate device
memory (application-owned memory budgets, fixed-footprint deployments).  It must give
the same d u~/dt as esd_rhs, call after call, from its fixed scratch array, and reject
meshes larger than that array before launching anything.

Collected last on purpose (file name), so a failure here stops a -x run only after every
other test has run."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup(dim, M, p, state):
    import esd_inputs as I
    import paper_2312_07874_gb300 as E
    mesh, X = I.config_mesh(dim, M, 2 * np.pi, p, True)
    gm = E.Mesh(dim, p, X, mesh.nbr_elem, mesh.nbr_face, flux="LF")
    x = gm.volume_nodes()
    f = I.config_state_fn(dim, 2 * np.pi, state)
    return gm, np.ascontiguousarray(np.transpose(f(x), (0, 2, 1)))


@pytest.mark.parametrize("dim,M,p,state", [(3, 3, 3, "tgv"), (2, 8, 4, "vortex")])
def test_static_scratch_matches_rhs_on_consecutive_calls(dim, M, p, state):
    import torch
    import paper_2312_07874_gb300 as E
    gm, un = _setup(dim, M, p, state)
    u0 = gm.l2_project(torch.from_numpy(un).cuda())
    rng = np.random.default_rng(21)
    u1 = u0 + 1e-3 * torch.from_numpy(rng.standard_normal(tuple(u0.shape))).cuda()
    for u in (u0, u1):                       # two calls in a row, different inputs
        ref = torch.empty_like(u)
        got = torch.full_like(u, float("nan"))
        st = E.lib().esd_rhs(gm.handle, E._ptr(u), E._ptr(ref), None)
        assert st == 0
        st = E.lib().esd_rhs_static_scratch(gm.handle, E._ptr(u), E._ptr(got), None)
        assert st == 0, E.lib().esd_last_error()
        torch.cuda.synchronize()
        gm.check()
        scale = ref.abs().amax(dim=(0, 2))
        err = (got - ref).abs().amax(dim=(0, 2)) / scale
        assert torch.all(err < 1e-12), err


def test_static_scratch_rejects_meshes_beyond_its_limit():
    import torch
    import paper_2312_07874_gb300 as E
    gm, un = _setup(3, 8, 4, "tgv")          # 3072 tets at p = 4 need ~47 MB of scratch
    u = gm.l2_project(torch.from_numpy(un).cuda())
    out = torch.zeros_like(u)
    st = E.lib().esd_rhs_static_scratch(gm.handle, E._ptr(u), E._ptr(out), None)
    assert st == -7
    assert b"limited to" in E.lib().esd_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0     # nothing was launched


def test_static_scratch_after_device_reset():
    """The scratch array's device address is looked up on each call, so the entry point
    still matches esd_rhs after the process's context has been reset and the library's
    device code reloaded (run in a child process that uses no torch)."""
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "no_alloc_reset_child.py")
    r = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [l.split() for l in r.stdout.splitlines() if l.startswith("round")]
    assert len(lines) == 2, r.stdout
    for l in lines:
        assert all(float(e) < 1e-12 for e in l[3:]), l


def test_calls_on_another_current_device_are_rejected():
    """A mesh belongs to the device current at its creation; a compute call made while
    another device is current returns ESD_ERR_ARG before launching anything.  With one
    GPU the mismatch is made by overwriting the handle's recorded device (test hook)."""
    import torch
    import paper_2312_07874_gb300 as E
    gm, un = _setup(2, 4, 2, "vortex")
    u = gm.l2_project(torch.from_numpy(un).cuda())
    out = torch.zeros_like(u)
    dev = torch.cuda.current_device()
    assert E.lib().esd_debug_set_mesh_device(gm.handle, dev + 1) == 0
    for call in (E.lib().esd_rhs, E.lib().esd_rhs_static_scratch):
        assert call(gm.handle, E._ptr(u), E._ptr(out), None) == -1
        assert b"is current" in E.lib().esd_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0     # nothing was launched
    assert E.lib().esd_debug_set_mesh_device(gm.handle, dev) == 0
    assert E.lib().esd_rhs_static_scratch(gm.handle, E._ptr(u), E._ptr(out), None) == 0
    torch.cuda.synchronize()
    assert float(out.abs().max()) > 0.0
