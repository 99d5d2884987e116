"""Oracle evaluations run in worker processes by the GPU tests (the long-double reference is
slow on one core).  Each job receives a small region of the mesh -- the elements it needs,
with a local facet-neighbour table -- and returns numpy arrays.  The pool uses the 'spawn'
start method: a process forked after the parent's first CUDA call can hang."""
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np

_POOL = None


def pool():
    global _POOL
    if _POOL is None:
        n = max(1, min(16, (os.cpu_count() or 1)))
        _POOL = ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
    return _POOL


def region(nbr_elem, elems, rings):
    """(region, local nbr table, local indices of elems): ``elems`` and ``rings`` rings of
    facet neighbours around them; neighbours outside the region point to the element itself."""
    nbr_elem = np.asarray(nbr_elem)
    reg = np.unique(np.asarray(elems))
    for _ in range(rings):
        reg = np.unique(np.concatenate([reg, nbr_elem[reg].ravel()]))
    pos = np.minimum(np.searchsorted(reg, nbr_elem[reg]), len(reg) - 1)
    loc = np.where(reg[pos] == nbr_elem[reg], pos, np.arange(len(reg))[:, None])
    return reg, loc, np.searchsorted(reg, elems)


def rhs_job(dim, p, X, nbr, face, um, elems, flux, gamma, ext):
    """(d u~/dt, term scale) of ``elems`` in long double (ext) or FP64, on the given region."""
    from oracle import extended
    dtype = extended.EXT if ext else np.float64
    Dx, need, local = extended.sub_discretization(dim, p, X, nbr, face, elems, flux, gamma, dtype)
    return Dx.rhs(np.asarray(um)[need].astype(dtype), "sparse", elems=local, return_scale=True)


def vjp_job(dim, p, X, nbr, face, um, cot, e, flux, gamma, ext):
    """(J^T cot) restricted to element e (local index), long double (ext) or FP64."""
    from oracle import extended
    from oracle.jacobian import local_vjp_batched
    dtype = extended.EXT if ext else np.float64
    nb = np.unique(np.concatenate([[e], nbr[e]]))
    ring = np.unique(np.concatenate([nb, nbr[nb].ravel()]))
    Dx, need, _ = extended.sub_discretization(dim, p, X, nbr, face, ring, flux, gamma, dtype)
    return local_vjp_batched(Dx, np.asarray(um)[need], np.asarray(cot)[need], int(np.searchsorted(need, e)))


def submit_rhs(D, X, um, elems, ext=True, per_job=1):
    """Futures of rhs_job over ``elems`` in order, ``per_job`` elements per job."""
    flux = "LF" if D.dissipation else "EC"
    elems = np.asarray(elems)
    futs = []
    for s in range(0, len(elems), per_job):
        grp = elems[s:s + per_job]
        reg, loc, le = region(D.geo.nbr_elem, grp, 2)
        futs.append(pool().submit(rhs_job, D.dim, D.p, np.asarray(X)[reg], loc, D.geo.nbr_face[reg],
                                  np.asarray(um)[reg], le, flux, D.gamma, ext))
    return futs


def submit_vjp(D, X, um, cot, elems, ext=True):
    flux = "LF" if D.dissipation else "EC"
    futs = []
    for e in np.asarray(elems):
        reg, loc, le = region(D.geo.nbr_elem, [e], 3)
        futs.append(pool().submit(vjp_job, D.dim, D.p, np.asarray(X)[reg], loc, D.geo.nbr_face[reg],
                                  np.asarray(um)[reg], np.asarray(cot)[reg], int(le[0]), flux, D.gamma, ext))
    return futs


def gather_rhs(futs):
    out = [f.result() for f in futs]
    return np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out])
