"""Sections 4.4-4.6, 5 and 6: the entropy-stable flux-differencing modal DSEM.

Oracle (test infrastructure only).  Three independent routes to the same
time derivative:

* ``rhs(..., route="dense")``: Eq. (entropy_stable) with explicit Hadamard
  products over all node pairs (full two-point-flux matrices of
  Eq. (two_point_flux_volume), Eq. (two_point_flux_facet), averaged metrics of
  Eq. (avg_vol_metrics), Eq. (avg_fac_metrics), facet correction of
  Eq. (facet_correction)), then Eq. (dudt_modal) with the weight-adjusted
  inverse of Eq. (weight_adjusted_inverse) (M = I).
* ``rhs(..., route="sparse")``: the paper's Section 5.1 algorithm: one
  directional flux per strictly-upper-triangular nonzero of each S^(l) with the
  direction {{2 g^(l)}}_ij of Eq. (avg_volume_metric), and one per nonzero of
  R^T B for the facet correction; it also counts flux evaluations
  (Eq. (num_fluxes)).
* ``rhs_hybridized``: Eq. (skew_hybridized) with the hybridized operators of
  Eq. (q_hybridized) and the split-form physical operators of
  Eq. (phys_hybridized).  The facet term there is read as premultiplied by V^T
  (it is a nodal vector in the print, added to a modal one).

The entropy projection is Eq. (entropy_expansion) (equivalently
Eq. (matvec_entropy_projection)); the interface flux is Eq. (interface_flux)
with Eq. (num_flux).  Modal states use the ABI layout [n_elem, N_c, N_p*].
"""
import numpy as np
from .reference import RefElement
from .pkd import vandermonde
from .geometry import Geometry
from . import euler


class Discretization:
    """The discretisation of one mesh, in floating-point type ``dtype`` (FP64 by default;
    np.longdouble for the extended-precision evaluation).  ``perm``: the facet-node
    permutations, when known (otherwise found by matching facets); ``unmatched``: facets
    whose neighbour is outside this (sub-)mesh (see Geometry)."""

    def __init__(self, dim, p, map_nodes, nbr_elem, nbr_face, flux="LF", gamma=euler.GAMMA,
                 dtype=float, perm=None, unmatched=None):
        self.dim, self.p = dim, p
        self.dtype = np.dtype(dtype).type
        self.ref = RefElement(dim, p, self.dtype)
        self.V = vandermonde(self.ref, p)
        self.geo = Geometry(self.ref, map_nodes, nbr_elem, nbr_face, perm=perm, unmatched=unmatched)
        self.dissipation = (flux == "LF")
        self.gamma = gamma
        self.Np = self.V.shape[1]
        self.Nc = dim + 2
        self.E = self.geo.E

    # ---- linear operators ---------------------------------------------------------
    def to_nodal(self, um):
        """u = V u~  (Eq. (modal_to_nodal)); [E, Nc, Np] -> [E, Nq, Nc]."""
        return np.einsum("ij,ecj->eic", self.V, um)

    def minv(self, y, elems):
        """Weight-adjusted inverse mass matrix V^T W J^-1 V applied to modal y [e, Np, Nc]."""
        ref, J = self.ref, self.geo.J_vol[elems]
        t = np.einsum("ij,ejc->eic", self.V, y)
        t = (ref.w[None, :] / J)[..., None] * t
        return np.einsum("ij,eic->ejc", self.V, t)

    def project_entropy(self, um, elems=None):
        """w~ of Eq. (entropy_expansion): M~^-1 V^T W J W(V u~); returns [e, Np, Nc]."""
        elems = np.arange(self.E) if elems is None else elems
        u = self.to_nodal(um[elems])
        wn = euler.entropy_vars(u, self.gamma)
        t = np.einsum("ij,eic->ejc", self.V, (self.ref.w[None, :] * self.geo.J_vol[elems])[..., None] * wn)
        return self.minv(t, elems)

    def states(self, um, need=None):
        """Entropy-projected conservative states at volume and facet nodes (Eq. (entropy_variables)).

        ``need`` restricts the work to a subset of elements (the others are left at a
        harmless admissible placeholder and must not be read)."""
        if need is not None:
            need = np.asarray(need)
            sub_um = um[need]
            wt = self.project_entropy(um, need)
            w = np.einsum("ij,ejc->eic", self.V, wt)
            wf = [np.einsum("ji,eic->ejc", R, w) for R in self.ref.R]
            full = lambda x: np.broadcast_to(x[:1], (self.E,) + x.shape[1:]).copy()
            Ut = full(euler.cons_from_entropy(w, self.gamma))
            Ut[need] = euler.cons_from_entropy(w, self.gamma)
            Utf = []
            for x in wf:
                y = euler.cons_from_entropy(x, self.gamma)
                z = full(y)
                z[need] = y
                Utf.append(z)
            W = full(w)
            W[need] = w
            del sub_um
            return W, Ut, Utf
        wt = self.project_entropy(um)
        w = np.einsum("ij,ejc->eic", self.V, wt)
        wf = [np.einsum("ji,eic->ejc", R, w) for R in self.ref.R]
        Ut = euler.cons_from_entropy(w, self.gamma)
        Utf = [euler.cons_from_entropy(x, self.gamma) for x in wf]
        return w, Ut, Utf

    # ---- residual -------------------------------------------------------------------
    def interface_fluxes(self, Utf, elems):
        geo = self.geo
        out = []
        for z in range(self.ref.Nf):
            e2 = geo.nbr_elem[elems, z]
            z2 = geo.nbr_face[elems, z]
            ext = np.stack([Utf[z2[k]][e2[k]][geo.perm[elems[k], z]] for k in range(len(elems))])
            out.append(euler.interface_flux(Utf[z][elems], ext, geo.n_fac[z][elems], self.dissipation, self.gamma))
        return out

    def nodal_residual(self, um, route="dense", elems=None, chunk=16, return_count=False,
                       return_scale=False):
        """r of Eq. (entropy_stable) for the elements ``elems``: [e, Nq, Nc].

        ``return_scale`` (sparse route): also return, per node and variable, the sum of the
        absolute values of the terms that r adds up (every pair flux times its operator
        entry, every facet-correction term, every lifted interface-flux term)."""
        if elems is None:
            elems = np.arange(self.E)
            w, Ut, Utf = self.states(um)
        else:
            elems = np.asarray(elems)
            need = np.unique(np.concatenate([elems, self.geo.nbr_elem[elems].ravel()]))
            w, Ut, Utf = self.states(um, need if len(need) < self.E else None)
        out, scales = [], []
        count = 0
        for s in range(0, len(elems), chunk):
            el = elems[s:s + chunk]
            fstar = self.interface_fluxes(Utf, el)
            if route == "dense":
                r = self._residual_dense(el, Ut, Utf, fstar)
            elif route == "sparse":
                r, count, T = self._residual_sparse(el, Ut, Utf, fstar, return_scale)
                scales.append(T)
            else:
                raise ValueError(route)
            out.append(r)
        r = np.concatenate(out, axis=0)
        if return_scale:
            return r, np.concatenate(scales, axis=0)
        return (r, count) if return_count else r

    def _residual_dense(self, el, Ut, Utf, fstar):
        ref, geo, d = self.ref, self.geo, self.dim
        U = Ut[el]
        G = geo.G_vol[el]
        F = [euler.ranocha_flux(U[:, :, None, :], U[:, None, :, :], m, self.gamma) for m in range(d)]
        r = np.zeros(U.shape, dtype=U.dtype)
        for l in range(d):
            acc = sum(0.5 * (G[:, :, None, l, m] + G[:, None, :, l, m])[..., None] * F[m] for m in range(d))
            r -= np.einsum("ij,eijc->eic", 2.0 * ref.S[l], acc)
        for z in range(ref.Nf):
            Uf = Utf[z][el]
            JnV = np.einsum("eilm,l->eim", G, ref.nhat[z])
            JnF = geo.Jn_fac[z][el]
            Ff = [euler.ranocha_flux(U[:, :, None, :], Uf[:, None, :, :], m, self.gamma) for m in range(d)]
            acc = sum(0.5 * (JnV[:, :, None, m] + JnF[:, None, :, m])[..., None] * Ff[m] for m in range(d))
            RtB = ref.R[z].T @ ref.B[z]
            C = RtB[None, :, :, None] * acc
            C1, Ct1 = C.sum(axis=2), C.sum(axis=1)
            g = (ref.wf[z][None, :] * geo.Jf[z][el])[..., None] * fstar[z] - Ct1
            r -= C1 + np.einsum("ji,ejc->eic", ref.R[z], g)
        return r

    def _residual_sparse(self, el, Ut, Utf, fstar, want_scale=False):
        ref, geo, d = self.ref, self.geo, self.dim
        U = Ut[el]
        G = geo.G_vol[el]
        vol = np.zeros(U.shape, dtype=U.dtype)
        T = np.zeros(U.shape, dtype=U.dtype)           # sums of |terms| (want_scale)
        count = 0
        for l in range(d):
            I, J = np.nonzero(np.triu(ref.S[l], 1))
            for i, j in zip(I, J):
                g = G[:, i, l, :] + G[:, j, l, :]
                F = euler.ranocha_flux_dir(U[:, i], U[:, j], g, self.gamma)
                vol[:, i] += ref.S[l][i, j] * F
                vol[:, j] -= ref.S[l][i, j] * F
                if want_scale:
                    a = np.abs(ref.S[l][i, j] * F)
                    T[:, i] += a
                    T[:, j] += a
                count += 1
        r = -vol
        for z in range(ref.Nf):
            Uf = Utf[z][el]
            JnV = np.einsum("eilm,l->eim", G, ref.nhat[z])
            JnF = geo.Jn_fac[z][el]
            RtB = ref.R[z].T @ ref.B[z]
            C1 = np.zeros(U.shape, dtype=U.dtype)
            Ct1 = np.zeros(Uf.shape, dtype=U.dtype)
            aC1 = np.zeros(U.shape, dtype=U.dtype)
            aCt1 = np.zeros(Uf.shape, dtype=U.dtype)
            I, J = np.nonzero(RtB)
            for i, j in zip(I, J):
                n = 0.5 * (JnV[:, i] + JnF[:, j])
                C = RtB[i, j] * euler.ranocha_flux_dir(U[:, i], Uf[:, j], n, self.gamma)
                C1[:, i] += C
                Ct1[:, j] += C
                if want_scale:
                    aC1[:, i] += np.abs(C)
                    aCt1[:, j] += np.abs(C)
                count += 1
            bjf = (ref.wf[z][None, :] * geo.Jf[z][el])[..., None] * fstar[z]
            g = bjf - Ct1
            r -= C1 + np.einsum("ji,ejc->eic", ref.R[z], g)
            if want_scale:
                T += aC1 + np.einsum("ji,ejc->eic", np.abs(ref.R[z]), np.abs(bjf) + aCt1)
        return r, count, T

    def term_scale(self, um, elems):
        """Scale of the rounding of d u~/dt: the sums of |terms| of the nodal residual
        (nodal_residual(return_scale=True)) carried through |V|^T, |V| diag(W/J) |V|^T
        of Eq. (dudt_modal): [e, Nc, Np], an upper bound of |d u~/dt| entry by entry."""
        elems = np.asarray(elems)
        _, T = self.nodal_residual(um, "sparse", elems, return_scale=True)
        return self._modal_scale(T, elems)

    def _modal_scale(self, T, elems):
        aV = np.abs(self.V)
        y = np.einsum("ij,eic->ejc", aV, T)
        t = np.einsum("ij,ejc->eic", aV, y) * (self.ref.w[None, :] / self.geo.J_vol[elems])[..., None]
        return np.transpose(np.einsum("ij,eic->ejc", aV, t), (0, 2, 1))

    def rhs(self, um, route="dense", elems=None, chunk=16, return_scale=False):
        """d u~/dt of Eq. (dudt_modal) in the ABI layout [e, Nc, Np].  With ``return_scale``
        (sparse route) also the term scale of each output (see term_scale)."""
        elems = np.arange(self.E) if elems is None else np.asarray(elems)
        r = self.nodal_residual(um, route, elems, chunk, return_scale=return_scale)
        if return_scale:
            r, T = r
        y = np.einsum("ij,eic->ejc", self.V, r)
        dudt = np.transpose(self.minv(y, elems), (0, 2, 1))
        return (dudt, self._modal_scale(T, elems)) if return_scale else dudt

    # ---- hybridized route (Section 6) -------------------------------------------------
    def rhs_hybridized(self, um, elems=None):
        ref, geo, d = self.ref, self.geo, self.dim
        elems = np.arange(self.E) if elems is None else np.asarray(elems)
        w, Ut, Utf = self.states(um)
        Nq, Nf, Nqf = ref.Nq, ref.Nf, ref.Nqf
        Nb = Nq + Nf * Nqf
        Qbar = []
        for l in range(d):
            Q = np.zeros((Nb, Nb), dtype=self.dtype)
            Q[:Nq, :Nq] = ref.S[l]
            for z in range(Nf):
                s = slice(Nq + z * Nqf, Nq + (z + 1) * Nqf)
                Q[:Nq, s] = 0.5 * ref.nhat[z][l] * ref.R[z].T @ ref.B[z]
                Q[s, :Nq] = -0.5 * ref.nhat[z][l] * ref.B[z] @ ref.R[z]
                Q[s, s] = 0.5 * ref.nhat[z][l] * ref.B[z]
            Qbar.append(Q)
        Vbar = np.concatenate([self.V] + [R @ self.V for R in ref.R], axis=0)
        out = []
        for e in elems:
            Ubar = np.concatenate([Ut[e]] + [Utf[z][e] for z in range(Nf)], axis=0)
            Gbar = np.concatenate([geo.G_vol[e]] + [geo.G_fac[z][e] for z in range(Nf)], axis=0)
            vol = np.zeros(Ubar.shape, dtype=Ubar.dtype)
            for m in range(d):
                Qm = sum(0.5 * (Qbar[l] @ np.diag(Gbar[:, l, m]) + np.diag(Gbar[:, l, m]) @ Qbar[l]) for l in range(d))
                Fm = euler.ranocha_flux(Ubar[:, None, :], Ubar[None, :, :], m, self.gamma)
                vol += np.einsum("ij,ijc->ic", 2.0 * Qm, Fm)
            rhs = -Vbar.T @ vol
            fstar = self.interface_fluxes(Utf, np.array([e]))
            for z in range(Nf):
                fn = sum(geo.n_fac[z][e][:, m, None] * euler.euler_flux(Utf[z][e], m, self.gamma) for m in range(d))
                g = (ref.wf[z] * geo.Jf[z][e])[:, None] * (fstar[z][0] - fn)
                rhs -= (ref.R[z] @ self.V).T @ g
            out.append(rhs)
        y = np.stack(out)
        return np.transpose(self.minv(y, elems), (0, 2, 1))

    # ---- diagnostics (Theorems 2 and 4) ------------------------------------------------
    def conservation_rate(self, dudt):
        """sum_kappa 1^T W J V d u~/dt per conserved variable (left side of Eq. (conservation))."""
        y = np.einsum("ij,ecj->eic", self.V, dudt)
        return np.einsum("i,ei,eic->c", self.ref.w, self.geo.J_vol, y)

    def entropy_rate(self, um, dudt):
        """(d/dt sum 1^T W J s, sum of |terms|): the left side of Eq. (discrete_entropy_bound),
        sum_e (V^T W J W_e(V u~))^T d u~_e/dt, with the sum of absolute nodal terms for scale."""
        u = self.to_nodal(um)
        wn = euler.entropy_vars(u, self.gamma)
        y = np.einsum("ij,ecj->eic", self.V, dudt)
        terms = (self.ref.w[None, :] * self.geo.J_vol)[..., None] * wn * y
        return terms.sum(), np.abs(terms).sum()
