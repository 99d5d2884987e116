"""The oracle's time derivative evaluated in extended precision on a sample of elements.

Oracle (test infrastructure only).  This is the same discretisation as
oracle/residual.py -- Eq. (dudt_modal) with the nodal residual of Eq. (entropy_stable)
by the sparse route of Section 5.1, the entropy projection of Eq. (entropy_expansion)
and the interface flux of Eq. (num_flux) -- with every step carried out in
``np.longdouble`` from the FP64 inputs (modal state and mapping nodes, which convert
exactly): quadrature rules, operators, PKD basis, geometry, projection, fluxes and the
weight-adjusted inverse.  ``np.longdouble`` has a 64-bit significand on x86-64 (unit
roundoff 5.4e-20) and is IEEE binary128 on AArch64 (unit roundoff 9.6e-35); either way
the result is the exact value of the method at the given FP64 inputs to far better than
FP64 resolution, so it measures the FP64 error of any implementation, the oracle's own
included.

Only the sampled elements and their facet neighbours (whose traces enter the interface
flux) are built, as a sub-mesh; its facet-node permutations (integers) are taken from the
FP64 discretisation of the whole mesh, or matched within the sub-mesh
(sub_discretization, which serves in FP64 too when the whole mesh is too large to build).
"""
import numpy as np

from .residual import Discretization

EXT = np.longdouble


def submesh(nbr_elem, elems):
    """(need, local nbr table, local indices of elems): ``need`` = the sorted union of
    ``elems`` and their facet neighbours; neighbours outside ``need`` point to the element
    itself in the local table (they are never read: only ``elems`` get residuals)."""
    nbr_elem = np.asarray(nbr_elem)
    elems = np.asarray(elems)
    need = np.unique(np.concatenate([elems, nbr_elem[elems].ravel()]))
    pos = np.searchsorted(need, nbr_elem[need])
    pos = np.minimum(pos, len(need) - 1)
    inside = need[pos] == nbr_elem[need]
    own = np.broadcast_to(np.arange(len(need))[:, None], pos.shape)
    loc = np.where(inside, pos, own).astype(np.int64)
    return need, loc, np.searchsorted(need, elems)


def sub_discretization(dim, p, map_nodes, nbr_elem, nbr_face, elems, flux="LF", gamma=None,
                       dtype=EXT):
    """(discretisation of the sub-mesh around ``elems`` in type ``dtype``, need, local indices
    of elems), built from the mesh arrays alone (no geometry of the whole mesh): facets
    between two sub-mesh elements are matched as usual, the outer facets of the neighbours
    are left unmatched (never read)."""
    need, loc, local = submesh(nbr_elem, elems)
    unmatched = loc == np.arange(len(need))[:, None]
    X = np.asarray(map_nodes, dtype=np.float64)[need].astype(dtype)
    kw = {} if gamma is None else dict(gamma=gamma)
    Dx = Discretization(dim, p, X, loc, np.asarray(nbr_face)[need], flux=flux, dtype=dtype,
                        unmatched=unmatched, **kw)
    return Dx, need, local


def discretization(D64, map_nodes, elems, dtype=EXT, flux=None):
    """The extended-precision discretisation of the sub-mesh around ``elems``, given the
    FP64 discretisation ``D64`` of the whole mesh (for its connectivity and permutations)."""
    need, loc, local = submesh(D64.geo.nbr_elem, elems)
    X = np.asarray(map_nodes, dtype=np.float64)[need].astype(dtype)
    flux = flux if flux is not None else ("LF" if D64.dissipation else "EC")
    Dx = Discretization(D64.dim, D64.p, X, loc, D64.geo.nbr_face[need], flux=flux,
                        gamma=D64.gamma, dtype=dtype, perm=D64.geo.perm[need])
    return Dx, need, local


def rhs(D64, map_nodes, um, elems, dtype=EXT):
    """d u~/dt of the sampled elements [len(elems), Nc, Np] in extended precision."""
    Dx, need, local = discretization(D64, map_nodes, elems, dtype)
    umx = np.asarray(um, dtype=np.float64)[need].astype(dtype)
    return Dx.rhs(umx, "sparse", elems=local)


def rhs_and_scale(D64, map_nodes, um, elems, dtype=EXT):
    """(d u~/dt, term scale) of the sampled elements in extended precision; the scale is
    Discretization.term_scale, the sums of |terms| carried through the modal transforms."""
    Dx, need, local = discretization(D64, map_nodes, elems, dtype)
    umx = np.asarray(um, dtype=np.float64)[need].astype(dtype)
    return Dx.rhs(umx, "sparse", elems=local, return_scale=True)


def project_entropy(D64, map_nodes, um, elems, dtype=EXT):
    """w~ of Eq. (entropy_expansion) for the sampled elements, [e, Np, Nc], extended precision."""
    Dx, need, local = discretization(D64, map_nodes, elems, dtype)
    umx = np.asarray(um, dtype=np.float64)[need].astype(dtype)
    return Dx.project_entropy(umx, local)


def local_vjp(D64, map_nodes, um, cot, e, dtype=EXT):
    """(J^T cot) restricted to the modes of element e (oracle.jacobian.local_vjp_batched) in
    extended precision, on the sub-mesh of e's neighbours and their neighbours."""
    from .jacobian import local_vjp_batched
    nbr = D64.geo.nbr_elem
    nb = np.unique(np.concatenate([[e], nbr[e]]))
    ring = np.unique(np.concatenate([nb, nbr[nb].ravel()]))
    Dx, need, _ = discretization(D64, map_nodes, ring, dtype)
    return local_vjp_batched(Dx, np.asarray(um)[need], np.asarray(cot)[need], int(np.searchsorted(need, e)))
