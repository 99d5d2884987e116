"""Failure detection on the GPU without a fault: the kernels' bounded waits give up,
report through the mesh's flag, and leave the context usable."""
import numpy as np
import pytest

from gpu_common import workload, gpu_mesh, to_dev

pytestmark = pytest.mark.gpu


def test_staging_wait_times_out_and_context_survives():
    import torch
    import paper_2312_07874_gb300 as E
    mesh, X, D, um = workload(3, 3, 2, True, "LF", "density_wave")
    gm = gpu_mesh(3, 2, X, mesh)
    u = to_dev(um)
    before = gm.rhs(u)
    gm.check()
    E.esd_debug_staging_timeout(gm.handle, 0.05)
    with pytest.raises(E.EsdError) as ex:
        gm.check()
    assert ex.value.status == -5          # ESD_ERR_TIMEOUT
    gm.check()                            # the flag was cleared by the report
    after = gm.rhs(u)                     # the context still runs kernels
    torch.cuda.synchronize()
    gm.check()
    assert torch.equal(before, after)
