"""Sections 4.1-4.2 and 4.5-4.6: polynomial mapping, metric terms, Nanson
normals, interpolated Jacobian determinant, and facet matching.

Oracle (test infrastructure only).

* Mapping (Eq. (poly_mapping)): degree-p_g Lagrange interpolation through the
  caller's mapping nodes, which sit on the equispaced degree-p_g lattice of the
  reference simplex (first lattice index fastest); the Lagrange polynomials of
  that lattice have a closed product form in barycentric coordinates.
* Metrics: exact adjugate in 2D; in 3D the conservative curl form of
  Eq. (metric_interpolants), Eq. (conservative_curl) with degree-(q+1)
  interpolation on the equispaced lattice, reading the three curls as the
  COLUMNS m = 1, 2, 3 of G_lm = J d xi_l / d x_m (for which G equals the
  adjugate whenever the interpolation is exact).  Mapping-node positions are
  translated by the element's first mapping node before the interpolants are
  formed (and before any gradient is taken); the curl of the interpolant of
  c * grad x_k and the gradient of a constant vanish identically, so this
  changes nothing but rounding.
* Facet normals and J^(kappa,zeta): Eq. (nanson).
* J used with W (mass matrix, projection): the degree-p_g interpolant of
  det(grad x) at the mapping nodes, Eq. (jacobian_approx).
* Facet matching (Assumption 2): for each facet the neighbour's node order is
  the identity or the reversal of the first facet coordinate; the one for which
  physical node positions differ by one constant vector (the periodic shift) is
  taken, and equal/opposite normals and equal weighted areas are verified.
"""
import numpy as np

from .jacobi import _working_type


def lattice(dim, P, dtype=float):
    """The equispaced degree-P lattice -1 + 2 i/P, first index fastest, in type ``dtype``."""
    T = np.dtype(dtype).type
    c = lambda i: T(-1) + T(2 * i) / T(P)
    pts = []
    if dim == 2:
        for j in range(P + 1):
            for i in range(P + 1 - j):
                pts.append((c(i), c(j)))
    else:
        for k in range(P + 1):
            for j in range(P + 1 - k):
                for i in range(P + 1 - j - k):
                    pts.append((c(i), c(j), c(k)))
    return np.array(pts, dtype=T)


def _barycentric(xi):
    """Barycentric coordinates of reference-simplex points, lambda_{k+1} = (xi_k + 1)/2 and
    lambda_1 = 1 - sum_k lambda_{k+1}, with d lambda / d xi as a constant matrix."""
    xi = np.atleast_2d(xi)
    dim = xi.shape[1]
    lam = np.concatenate([1.0 - (xi + 1.0).sum(1, keepdims=True) / 2.0, (xi + 1.0) / 2.0], axis=1)
    dlam = np.zeros((dim + 1, dim), dtype=xi.dtype)
    dlam[0, :] = -0.5
    for k in range(dim):
        dlam[k + 1, k] = 0.5
    return lam, dlam


def lagrange_simplex(dim, P, targets):
    """L[t, i] = ell_i(x_t), dL[t, i, k] = d ell_i / d xi_k (x_t) for the degree-P equispaced lattice.

    Closed form for the equispaced simplex lattice: the node with barycentric
    index (I_0..I_d) (sum P) has ell = prod_k prod_{m < I_k} (P lambda_k - m)/(I_k - m),
    which vanishes at every other lattice node and is 1 at its own.
    """
    nodes = lattice(dim, P)
    lam_n, _ = _barycentric(nodes)
    Ibar = np.rint(lam_n * P).astype(int)                       # [n, d+1]
    F = _working_type(targets)
    lam, dlam = _barycentric(np.asarray(targets, dtype=F))      # [t, d+1]
    T, n = lam.shape[0], len(nodes)
    L = np.ones((T, n), dtype=F)
    dLdlam = np.zeros((T, n, dim + 1), dtype=F)
    for i in range(n):
        fac = []
        for k in range(dim + 1):
            f = np.ones(T, dtype=F)
            df = np.zeros(T, dtype=F)
            for m in range(Ibar[i, k]):
                term = (P * lam[:, k] - m) / (Ibar[i, k] - m)
                df = df * term + f * P / (Ibar[i, k] - m)
                f = f * term
            fac.append((f, df))
        for k in range(dim + 1):
            L[:, i] *= fac[k][0]
            g = fac[k][1].copy()
            for k2 in range(dim + 1):
                if k2 != k:
                    g *= fac[k2][0]
            dLdlam[:, i, k] = g
    dL = np.einsum("tik,ks->tis", dLdlam, dlam)
    return L, dL


def _det(A):
    """Determinant of the trailing 2x2 or 3x3 blocks, by cofactors (any float type)."""
    if A.shape[-1] == 2:
        return A[..., 0, 0] * A[..., 1, 1] - A[..., 0, 1] * A[..., 1, 0]
    return (A[..., 0, 0] * (A[..., 1, 1] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 1])
            - A[..., 0, 1] * (A[..., 1, 0] * A[..., 2, 2] - A[..., 1, 2] * A[..., 2, 0])
            + A[..., 0, 2] * (A[..., 1, 0] * A[..., 2, 1] - A[..., 1, 1] * A[..., 2, 0]))


class Geometry:
    """Per-element geometric factors of a mesh of curved simplices, in the floating-point
    type of the reference element.  ``perm`` (the facet-node permutations, integers) may be
    given instead of being found by matching facets.  ``unmatched`` ([E, N_f] bool) marks
    facets whose neighbour is not part of this (sub-)mesh: they are not matched and their
    permutation (the identity) must not be used."""

    def __init__(self, ref, map_nodes, nbr_elem, nbr_face, pg=None, perm=None, unmatched=None):
        self.ref = ref
        dim, q = ref.dim, ref.q
        X = np.asarray(map_nodes, dtype=ref.dtype)      # [E, N*_pg, dim]
        E = X.shape[0]
        npg = X.shape[1]
        pg = pg if pg is not None else next(P for P in range(1, 40)
                                            if len(lattice(dim, P)) == npg)
        self.pg = pg
        self.E = E
        # points where geometry is needed: volume nodes then all facet nodes
        pts = np.concatenate([ref.xi] + ref.xif, axis=0)
        Lm, dLm = lagrange_simplex(dim, pg, pts)
        x = np.einsum("ti,eid->etd", Lm, X)
        Xl = X - X[:, :1, :]                             # element-local translation (see header)
        A = np.einsum("tik,eim->etmk", dLm, Xl)         # A[e,t,m,k] = d x_m / d xi_k
        self.x_vol = x[:, :ref.Nq]
        self.x_fac = [x[:, ref.Nq + z * ref.Nqf: ref.Nq + (z + 1) * ref.Nqf] for z in range(ref.Nf)]
        if dim == 2:
            G = np.empty(A.shape, dtype=A.dtype)
            G[..., 0, 0] = A[..., 1, 1]
            G[..., 0, 1] = -A[..., 0, 1]
            G[..., 1, 0] = -A[..., 1, 0]
            G[..., 1, 1] = A[..., 0, 0]
        else:
            G = self._curl_metrics(X, pg, pts)
        self.G_all = G                                   # [E, npts, l, m]
        self.G_vol = G[:, :ref.Nq]
        self.G_fac = [G[:, ref.Nq + z * ref.Nqf: ref.Nq + (z + 1) * ref.Nqf] for z in range(ref.Nf)]
        # Nanson: J^(k,z) n = G^T nhat
        self.Jn_fac = [np.einsum("etlm,l->etm", self.G_fac[z], ref.nhat[z]) for z in range(ref.Nf)]
        self.Jf = [np.linalg.norm(v, axis=-1) for v in self.Jn_fac]
        self.n_fac = [self.Jn_fac[z] / self.Jf[z][..., None] for z in range(ref.Nf)]
        # interpolated Jacobian determinant (degree pg) at volume nodes
        lat = lattice(dim, pg, ref.dtype)
        _, dLl = lagrange_simplex(dim, pg, lat)
        Al = np.einsum("tik,eim->etmk", dLl, Xl)
        detl = _det(Al)
        Lv, _ = lagrange_simplex(dim, pg, ref.xi)
        self.J_vol = np.einsum("ti,ei->et", Lv, detl)
        self.J_exact_vol = _det(A[:, :ref.Nq])
        self.det_lattice = detl
        self.nbr_elem = np.asarray(nbr_elem)
        self.nbr_face = np.asarray(nbr_face)
        if perm is None:
            self._match_facets(unmatched)
        else:
            self.perm = np.asarray(perm, dtype=np.int64)

    def _curl_metrics(self, X, pg, pts):
        ref = self.ref
        dim, q = ref.dim, ref.q
        Xl = X - X[:, :1, :]                              # element-local translation
        inodes = lattice(dim, q + 1, ref.dtype)
        Lm_i, dLm_i = lagrange_simplex(dim, pg, inodes)
        xi_ = np.einsum("ti,eid->etd", Lm_i, Xl)          # x at interpolation nodes
        gi = np.einsum("tik,eim->etmk", dLm_i, Xl)        # grad_xi x_m at interpolation nodes
        r1 = xi_[..., 2:3] * gi[..., 1, :]                # x3 grad x2
        r2 = xi_[..., 2:3] * gi[..., 0, :]                # x3 grad x1
        r3 = xi_[..., 0:1] * gi[..., 1, :]                # x1 grad x2
        _, dLq = lagrange_simplex(dim, q + 1, pts)        # [t, i, k]
        def curl(r):                                      # sum_i grad ell_i x r_i
            return np.einsum("tik,eil->etkl", dLq, r)     # outer; take the antisymmetric part below
        out = np.empty((X.shape[0], len(pts), 3, 3), dtype=ref.dtype)
        for col, (r, sgn) in enumerate(((r1, -1.0), (r2, 1.0), (r3, 1.0))):
            T = curl(r)                                   # T[e,t,k,l] = sum_i d_k ell_i r_i,l
            c = np.stack([T[..., 1, 2] - T[..., 2, 1],
                          T[..., 2, 0] - T[..., 0, 2],
                          T[..., 0, 1] - T[..., 1, 0]], axis=-1)
            out[..., :, col] = sgn * c
        return out

    def _match_facets(self, unmatched=None):
        ref = self.ref
        n, dim = ref.q + 1, ref.dim
        if dim == 2:
            cands = [np.arange(n), np.arange(n)[::-1]]
        else:
            a = ref.alpha_f
            cands = [np.arange(n * n), (n - 1 - a[:, 0]) * n + a[:, 1]]
        self.perm = np.zeros((self.E, ref.Nf, ref.Nqf), dtype=np.int64)
        for e in range(self.E):
            for z in range(ref.Nf):
                if unmatched is not None and unmatched[e, z]:
                    self.perm[e, z] = cands[0]
                    continue
                e2, z2 = int(self.nbr_elem[e, z]), int(self.nbr_face[e, z])
                xa, xb = self.x_fac[z][e], self.x_fac[z2][e2]
                scale = np.max(np.abs(xa - xa.mean(0))) + 1e-300
                found = None
                for c in cands:
                    d = xa - xb[c]
                    if np.max(np.abs(d - d[0])) < 1e-9 * scale:
                        found = c
                        break
                if found is None:
                    raise ValueError(f"facet {z} of element {e} does not match its neighbour")
                na, nb = self.n_fac[z][e], self.n_fac[z2][e2][found]
                wa = ref.wf[z] * self.Jf[z][e]
                wb = ref.wf[z2][found] * self.Jf[z2][e2][found]
                if np.max(np.abs(na + nb)) > 1e-8 or np.max(np.abs(wa - wb)) > 1e-8 * np.max(np.abs(wa)):
                    raise ValueError(f"facet {z} of element {e}: normals/weights do not match")
                self.perm[e, z] = found
