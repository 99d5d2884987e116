"""Accuracy of the table-driven log and exp used by the projection kernel, against
CUDA's own log/exp (torch on the GPU) and numpy on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs_log():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        np.exp(rng.uniform(-30, 30, 200000)),              # many octaves
        1.0 + rng.uniform(-1e-3, 1e-3, 100000),             # near 1 (the k = 0 / k = -1 seams)
        rng.uniform(0.5, 2.0, 100000),
        np.array([1.0, 2.0, 0.5, 1.0 + 2**-52, 1.0 - 2**-53, 71.42857142857143, 1.0 / 71.4]),
    ])
    return x


def _inputs_exp():
    rng = np.random.default_rng(1)
    return np.concatenate([rng.uniform(-50, 50, 200000), rng.uniform(-1e-3, 1e-3, 100000),
                           np.array([0.0, 1.0, -1.0, np.log(2.0), 20.0, -20.0])])


@pytest.mark.parametrize("which", [0, 1])
def test_table_math_accuracy(which):
    import torch
    import paper_2312_07874_gb300 as E
    x = _inputs_log() if which == 0 else _inputs_exp()
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    E.esd_debug_math(which, xd, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    ref_np = np.log(x) if which == 0 else np.exp(x)
    ref_cuda = (torch.log(xd) if which == 0 else torch.exp(xd)).cpu().numpy()
    if which == 0:
        # error relative to the result's magnitude, with an absolute floor at the seam x ~ 1
        scale = np.maximum(np.abs(ref_np), np.abs(x - 1.0))
    else:
        scale = np.abs(ref_np)
    # ln 1 = 0 exactly: there the absolute error itself must vanish
    scale = np.where(scale > 0.0, scale, 1.0)
    err_np = np.abs(got - ref_np) / scale
    err_cuda = np.abs(ref_cuda - ref_np) / scale
    eps = np.finfo(float).eps
    assert err_np.max() <= 2.0 * eps, err_np.max() / eps
    # no worse than CUDA's own implementation by more than one unit roundoff
    assert err_np.max() <= err_cuda.max() + eps
