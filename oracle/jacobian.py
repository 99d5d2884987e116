"""Complex-step Jacobian-vector products of the oracle's d u~/dt (not in the paper; the
reference for the hand-written adjoint).  Oracle (test infrastructure only).  The
element-local Jacobian transpose comes column by column (local_vjp) or with all columns
in one batched evaluation (local_vjp_batched, which also runs in long double).

For a real-analytic f, f(u + i h v) = f(u) + i h J v + O(h^2), so Im f(u + i h v) / h
gives J v exact to rounding for tiny h (no subtraction).  The max and |.| of the Davis
wave speed are continued through the real part of their arguments, i.e. the one-sided
derivative with ties resolved to the interior side -- the reading used by the adjoint.
"""
import copy

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


def _tiled(D, need, K):
    """A discretisation of K independent copies of the sub-mesh ``need`` of D (elements
    need[i] of copy k become element k*len(need) + i); facet neighbours outside ``need``
    point to the element itself and must not be read.  Geometry is copied, not rebuilt."""
    n = len(need)
    pos = np.searchsorted(need, D.geo.nbr_elem[need])
    pos = np.minimum(pos, n - 1)
    loc = np.where(need[pos] == D.geo.nbr_elem[need], pos, np.arange(n)[:, None])
    T = copy.copy(D)
    g = T.geo = copy.copy(D.geo)
    rep = lambda a: np.concatenate([a[need]] * K, axis=0)
    g.J_vol, g.G_vol, g.perm, g.nbr_face = rep(D.geo.J_vol), rep(D.geo.G_vol), rep(D.geo.perm), rep(D.geo.nbr_face)
    g.Jn_fac = [rep(a) for a in D.geo.Jn_fac]
    g.Jf = [rep(a) for a in D.geo.Jf]
    g.n_fac = [rep(a) for a in D.geo.n_fac]
    g.nbr_elem = np.concatenate([loc + k * n for k in range(K)], axis=0)
    T.E = g.E = n * K
    return T


def local_vjp_batched(D, um, cot, e):
    """(J^T cot) restricted to the modes of element e, as local_vjp, with all N_c N_p*
    complex-step directions in one evaluation: the elements whose d u~/dt depends on e's
    modes (e and its facet neighbours) are evaluated on N_c N_p* independent copies of
    their neighbourhood, copy k carrying the step i H in mode k of e.  Works in the
    discretisation's floating-point type (complex of it for the step)."""
    nb = np.unique(np.concatenate([[e], D.geo.nbr_elem[e]]))
    need = np.unique(np.concatenate([nb, D.geo.nbr_elem[nb].ravel()]))
    n, K = len(need), D.Nc * D.Np
    T = _tiled(D, need, K)
    ctype = np.result_type(D.dtype, np.complex64)
    U = np.concatenate([np.asarray(um)[need].astype(ctype)] * K, axis=0)
    ie = int(np.searchsorted(need, e))
    for k in range(K):
        c, j = divmod(k, D.Np)
        U[k * n + ie, c, j] += 1j * H
    inb = np.searchsorted(need, nb)
    targets = np.concatenate([k * n + inb for k in range(K)])
    col = np.imag(T.rhs(U, "sparse", elems=targets, chunk=len(targets))) / H
    col = col.reshape(K, len(nb), D.Nc, D.Np)
    return np.einsum("kbcj,bcj->k", col, np.asarray(cot)[nb]).reshape(D.Nc, D.Np)
