"""Section 3: tensor-product SBP operators in collapsed coordinates on the
reference triangle (Section 3.1) and tetrahedron (Section 3.2).

Oracle (test infrastructure only).  Every operator is assembled as a dense
matrix entry by entry from the printed formulas:

* collapsed maps: Eq. (tri_mapping); Eq. (tet_mapping) read with the third
  factor (1 - eta_3) in the first component (the print repeats (1 - eta_2));
* volume rules: Eq. (tri_quadrature), Eq. (tet_quadrature);
* facet rules: Eq. (tri_facet_quadrature_nodes), Eq. (tet_facet_quadrature_nodes),
  Eq. (tet_facet_quadrature_weights);
* derivative operators: Eq. (d_2d), Eq. (d_3d) read with delta_{alpha3 beta3}
  where the print has delta_{alpha3 alpha3};
* extrapolation operators: Eq. (r_2d), Eq. (r_3d);
* Q = W D, S = (Q - Q^T)/2, E = sum_zeta nhat R^T B R  (Definition 2, Eq. (e_decomp)).

Volume nodes are ordered by the multi-index alpha with alpha_1 slowest;
facet nodes of a tetrahedron by (alpha_1, alpha_2) with alpha_1 slowest.
"""
import itertools
import numpy as np
from .jacobi import gauss_jacobi, lagrange, lagrange_deriv, _working_type


def collapse(eta):
    """chi(eta): square -> reference triangle, cube -> reference tetrahedron."""
    eta = np.asarray(eta, dtype=_working_type(eta))
    if eta.shape[-1] == 2:
        e1, e2 = eta[..., 0], eta[..., 1]
        return np.stack([0.5 * (1 + e1) * (1 - e2) - 1.0, e2], axis=-1)
    e1, e2, e3 = eta[..., 0], eta[..., 1], eta[..., 2]
    return np.stack([0.25 * (1 + e1) * (1 - e2) * (1 - e3) - 1.0,
                     0.5 * (1 + e2) * (1 - e3) - 1.0,
                     e3], axis=-1)


class RefElement:
    """Reference simplex with tensor-product SBP operators of degree q (q1 = q2 (= q3) = qf = q),
    built in floating-point type ``dtype`` (FP64 by default)."""

    def __init__(self, dim, q, dtype=float):
        self.dim, self.q = dim, q
        self.dtype = T = np.dtype(dtype).type
        n = q + 1
        # 1D rules: LG in eta1, eta2 (and on facets); Gauss-Jacobi(1,0) in eta3
        self.r = [gauss_jacobi(q, 0, 0, T), gauss_jacobi(q, 0, 0, T)]
        if dim == 3:
            self.r.append(gauss_jacobi(q, 1, 0, T))
        self.alpha = np.array(list(itertools.product(range(n), repeat=dim)))   # alpha_1 slowest
        self.Nq = len(self.alpha)
        self.eta = np.stack([self.r[k][0][self.alpha[:, k]] for k in range(dim)], axis=-1)
        self.xi = collapse(self.eta)
        e = self.eta
        if dim == 2:
            self.w = 0.5 * (1 - e[:, 1]) * self.r[0][1][self.alpha[:, 0]] * self.r[1][1][self.alpha[:, 1]]
        else:
            self.w = ((1 - e[:, 1]) * (1 - e[:, 2]) / 8.0 * self.r[0][1][self.alpha[:, 0]]
                      * self.r[1][1][self.alpha[:, 1]] * self.r[2][1][self.alpha[:, 2]])
        self.W = np.diag(self.w)
        self._build_facets()
        self._build_derivatives()
        self.Q = [self.W @ D for D in self.D]
        self.S = [0.5 * (Q - Q.T) for Q in self.Q]
        self.E = [sum(self.nhat[z][l] * self.R[z].T @ self.B[z] @ self.R[z] for z in range(self.Nf))
                  for l in range(dim)]

    # ---- facets -------------------------------------------------------------------
    def _build_facets(self):
        q, n, dim, T = self.q, self.q + 1, self.dim, self.dtype
        etaLG, wLG = self.r[0]
        one, mone = np.array([1], dtype=T), np.array([-1], dtype=T)
        sqrt2, sqrt3 = np.sqrt(T(2)), np.sqrt(T(3))
        # 1D Lagrange values ell_beta(x) as [beta, t]
        l1 = lambda x: lagrange(self.r[0][0], x)
        l2 = lambda x: lagrange(self.r[1][0], x)
        self.xif, self.wf, self.R, self.nhat = [], [], [], []
        b = self.alpha
        if dim == 2:
            self.Nf, self.Nqf = 3, n
            i = np.arange(n)
            defs = [  # (eta of facet nodes, weight factor, nhat, R entries)
                (np.stack([etaLG, -np.ones(n, dtype=T)], -1), 1, np.array([0, -1], dtype=T),
                 l1(etaLG)[b[:, 0]][:, i].T * l2(mone)[b[:, 1], 0][None, :]),
                (np.stack([np.ones(n, dtype=T), etaLG], -1), sqrt2, np.array([1, 1], dtype=T) / sqrt2,
                 l1(one)[b[:, 0], 0][None, :] * l2(etaLG)[b[:, 1]][:, i].T),
                (np.stack([-np.ones(n, dtype=T), etaLG], -1), 1, np.array([-1, 0], dtype=T),
                 l1(mone)[b[:, 0], 0][None, :] * l2(etaLG)[b[:, 1]][:, i].T),
            ]
            for eta_f, fac, nh, R in defs:
                self.xif.append(collapse(eta_f))
                self.wf.append(fac * wLG)
                self.nhat.append(nh)
                self.R.append(R)
        else:
            self.Nf, self.Nqf = 4, n * n
            etaJ, wJ = self.r[2]
            l3 = lambda x: lagrange(etaJ, x)
            af = np.array(list(itertools.product(range(n), repeat=2)))     # (a1, a2), a1 slowest
            ef1, ef2 = etaLG[af[:, 0]], etaJ[af[:, 1]]
            wfac = wLG[af[:, 0]] * wJ[af[:, 1]]
            onesf = np.ones(len(af), dtype=T)
            half = T(1) / 2
            L1 = l1(etaLG)   # [beta, a]
            L2LG = l2(etaLG)
            L2J = l2(etaJ)   # LG basis in eta2 evaluated at GJ(1,0) nodes
            L3 = l3(etaJ)
            defs = [
                (np.stack([ef1, -onesf, ef2], -1), half, np.array([0, -1, 0], dtype=T),
                 L1[b[:, 0]][:, af[:, 0]].T * l2(mone)[b[:, 1], 0][None, :] * L3[b[:, 2]][:, af[:, 1]].T),
                (np.stack([onesf, ef1, ef2], -1), sqrt3 / 2, np.array([1, 1, 1], dtype=T) / sqrt3,
                 l1(one)[b[:, 0], 0][None, :] * L2LG[b[:, 1]][:, af[:, 0]].T * L3[b[:, 2]][:, af[:, 1]].T),
                (np.stack([-onesf, ef1, ef2], -1), half, np.array([-1, 0, 0], dtype=T),
                 l1(mone)[b[:, 0], 0][None, :] * L2LG[b[:, 1]][:, af[:, 0]].T * L3[b[:, 2]][:, af[:, 1]].T),
                (np.stack([ef1, ef2, -onesf], -1), half, np.array([0, 0, -1], dtype=T),
                 L1[b[:, 0]][:, af[:, 0]].T * L2J[b[:, 1]][:, af[:, 1]].T * l3(mone)[b[:, 2], 0][None, :]),
            ]
            self.alpha_f = af
            for eta_f, fac, nh, R in defs:
                self.xif.append(collapse(eta_f))
                self.wf.append(fac * wfac)
                self.nhat.append(nh)
                self.R.append(R)
        self.B = [np.diag(w) for w in self.wf]

    # ---- derivative operators -----------------------------------------------------
    def _build_derivatives(self):
        dim = self.dim
        A = self.alpha[:, None, :]   # row multi-index alpha
        Bm = self.alpha[None, :, :]  # column multi-index beta
        e1 = self.r[0][0][A[..., 0]]
        e2 = self.r[1][0][A[..., 1]]
        d1 = lagrange_deriv(self.r[0][0], self.r[0][0])   # [beta, alpha]: d ell_beta/d eta (eta_alpha)
        d2 = lagrange_deriv(self.r[1][0], self.r[1][0])
        dl1 = d1[Bm[..., 0], A[..., 0]]
        dl2 = d2[Bm[..., 1], A[..., 1]]
        dd = lambda k: (A[..., k] == Bm[..., k]).astype(self.dtype)
        if dim == 2:
            D1 = 2.0 / (1 - e2) * dl1 * dd(1)
            D2 = (1 + e1) / (1 - e2) * dl1 * dd(1) + dd(0) * dl2
            self.D = [D1, D2]
        else:
            e3 = self.r[2][0][A[..., 2]]
            d3 = lagrange_deriv(self.r[2][0], self.r[2][0])
            dl3 = d3[Bm[..., 2], A[..., 2]]
            D1 = 4.0 / ((1 - e2) * (1 - e3)) * dl1 * dd(1) * dd(2)
            D2 = (2 * (1 + e1) / ((1 - e2) * (1 - e3)) * dl1 * dd(1) * dd(2)
                  + 2.0 / (1 - e3) * dd(0) * dl2 * dd(2))
            D3 = (2 * (1 + e1) / ((1 - e2) * (1 - e3)) * dl1 * dd(1) * dd(2)
                  + (1 + e2) / (1 - e3) * dd(0) * dl2 * dd(2)
                  + dd(0) * dd(1) * dl3)
            self.D = [D1, D2, D3]
