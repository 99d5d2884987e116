"""Edge cases of the C ABI on the GPU: empty inputs, a ragged last element tile,
argument errors of the monitoring and batch entry points (all rejected before a launch)."""
import numpy as np
import pytest

from gpu_common import workload, gpu_mesh, to_dev, check_parity

pytestmark = pytest.mark.gpu


def test_empty_mesh_and_batch_rejected():
    import paper_2312_07874_gb300 as E
    with pytest.raises(E.EsdError) as ex:
        E.Mesh(3, 2, np.zeros((0, 10, 3)), np.zeros((0, 4), np.int32), np.zeros((0, 4), np.int8))
    assert ex.value.status == -1
    with pytest.raises(E.EsdError) as ex:
        E.esd_batch_create([])
    assert ex.value.status == -1


def test_ragged_last_tile_parity():
    """162 tetrahedra at 5 elements per CTA leave a last tile of 2: the parity of the whole
    output covers the partial tile (and the partial last warp of every tile)."""
    import torch
    mesh, X, D, um = workload(3, 3, 4, True, "LF", "density_wave")
    gm = gpu_mesh(3, 4, X, mesh)
    epc = gm.info["elems_per_cta_residual"]
    assert D.E % epc != 0, epc
    out = gm.rhs(to_dev(um))
    torch.cuda.synchronize()
    # the long-double sample includes the last element (in the partial tile)
    got = out.cpu().numpy()
    check_parity("ragged last tile", got, D, X, um, n_exact=4, seed=3)
    tail = np.arange(D.E - D.E % epc, D.E)
    check_parity("ragged last tile (tail)", got[tail], D, X, um, elems=tail, n_exact=len(tail))


def test_monitoring_arguments_rejected():
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(2, 3, 2)
    gm = gpu_mesh(2, 2, X, mesh)
    u = to_dev(um)
    host = np.zeros(16)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    assert E.lib().esd_integrals(gm.handle, E.ctypes.c_void_p(host.ctypes.data), E._ptr(out), None) == -1
    assert E.lib().esd_integrals(gm.handle, E._ptr(u), E.ctypes.c_void_p(host.ctypes.data), None) == -1
    assert E.lib().esd_integrals(None, E._ptr(u), E._ptr(out), None) == -1
    assert E.lib().esd_diagnostics(gm.handle, E._ptr(u), E.ctypes.c_void_p(host.ctypes.data), None) == -1
    assert E.lib().esd_debug_staging_timeout(gm.handle, 0.0, None) == -1
    gm.check()
