"""Complex-step Jacobian-vector products of the oracle's d u~/dt (not in the paper; the
reference for the hand-written adjoint).  Oracle (test infrastructure only).

For a real-analytic f, f(u + i h v) = f(u) + i h J v + O(h^2), so Im f(u + i h v) / h
gives J v exact to rounding for tiny h (no subtraction).  The max and |.| of the Davis
wave speed are continued through the real part of their arguments, i.e. the one-sided
derivative with ties resolved to the interior side -- the reading used by the adjoint.
"""
import numpy as np

H = 1e-30


def jvp(D, um, v, elems=None, route="sparse"):
    """J v of d u~/dt (all elements, or the listed ones) at the modal state um."""
    return np.imag(D.rhs(um + 1j * H * v, route, elems=elems)) / H


def rk4_jvp(D, um, v, dt, route="sparse"):
    from .timestep import rk4_step
    z = rk4_step(lambda x: D.rhs(x, route), um + 1j * H * v, dt)
    return np.imag(z) / H


def local_vjp(D, um, cot, e):
    """(J^T cot) restricted to the modes of element e, assembled column by column from
    complex-step Jacobian columns (only e and its facet neighbours depend on e's modes)."""
    nb = np.unique(np.concatenate([[e], D.geo.nbr_elem[e]]))
    out = np.zeros((D.Nc, D.Np))
    for c in range(D.Nc):
        for j in range(D.Np):
            v = np.zeros(um.shape)
            v[e, c, j] = 1.0
            col = jvp(D, um, v, elems=nb)
            out[c, j] = np.sum(cot[nb] * col)
    return out
