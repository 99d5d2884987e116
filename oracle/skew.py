"""Section 4.4: the conservative and skew-symmetric nodal SBP forms of the residual,
Eq. (rhs_cons) and Eq. (rhs_skew), with the modal update of Eq. (modal) through the
weight-adjusted inverse of Eq. (weight_adjusted_inverse).  Oracle (test infrastructure
only).

Unlike the entropy-stable scheme (oracle/residual.py), these forms evaluate the fluxes
f_m at the nodal solution u = V u~ itself (no entropy projection, no two-point flux):

  Eq. (rhs_cons):  r = sum_l Q^(l)T sum_m G^(l,m) f_m - sum_zeta R^T B J^zeta f*
  Eq. (rhs_skew):  r = 1/2 sum_l ( Q^(l)T sum_m G^(l,m) f_m - sum_m G^(l,m) Q^(l) f_m )
                       - sum_zeta R^T B J^zeta ( f* - 1/2 sum_m N^(zeta,m) R f_m )

with G^(l,m), J^zeta, N^(zeta,m) the diagonal matrices of Eq. (geometric_factors) (the
metric terms at the volume nodes, the facet scaling |G^T nhat| and the unit normal at the
facet nodes).  Both forms are written for any flux model: the compressible Euler
equations of Section 7.1 (interface flux Eq. (num_flux)), or scalar linear advection
f_m(u) = a_m u, the problem for which the skew-symmetric form was introduced (energy
stability on curved elements).

Operators (Q, R, B, W), geometry (G, J^zeta, n, the facet permutation) and the PKD
Vandermonde come from an oracle.residual.Discretization (in its floating-point type: FP64,
or long double for the extended-precision reference); the modal states use the ABI
layout [n_elem, N_c, N_p*].
"""
import numpy as np

from . import euler


class EulerModel:
    """Compressible Euler fluxes f_m (Eq. (euler)) and the interface flux of Eq. (num_flux)."""

    def __init__(self, dim, gamma=euler.GAMMA, dissipation=True):
        self.nc = dim + 2
        self.gamma = gamma
        self.dissipation = dissipation

    def flux(self, U, m):
        return euler.euler_flux(U, m, self.gamma)

    def numflux(self, UL, UR, n):
        return euler.interface_flux(UL, UR, n, self.dissipation, self.gamma)


class AdvectionModel:
    """Scalar linear advection u_t + div(a u) = 0 with constant a: f_m(u) = a_m u and the
    interface flux (a.n)(u^- + u^+)/2 - sigma |a.n| (u^+ - u^-)/2 (sigma = 0: central,
    sigma = 1: upwind)."""

    def __init__(self, a, upwind=False):
        self.a = np.asarray(a, dtype=float)
        self.nc = 1
        self.sigma = 1.0 if upwind else 0.0

    def flux(self, U, m):
        return self.a[m] * U

    def numflux(self, UL, UR, n):
        an = (n @ self.a)[..., None]
        return 0.5 * an * (UL + UR) - 0.5 * self.sigma * np.abs(an) * (UR - UL)


def nodal_states(D, um):
    """u = V u~ at the volume nodes [E, Nq, Nc] and its facet traces R^zeta u."""
    u = np.einsum("ij,ecj->eic", D.V, um)
    return u, [np.einsum("ji,eic->ejc", R, u) for R in D.ref.R]


def nodal_residual(D, um, model, form="skew", elems=None):
    """r of Eq. (rhs_skew) (form="skew") or Eq. (rhs_cons) (form="cons"): [e, Nq, Nc]."""
    if form not in ("skew", "cons"):
        raise ValueError(form)
    ref, geo, d = D.ref, D.geo, D.dim
    elems = np.arange(D.E) if elems is None else np.asarray(elems)
    u, uf = nodal_states(D, um)
    out = []
    for e in elems:
        G = geo.G_vol[e]
        f = [model.flux(u[e], m) for m in range(d)]
        r = np.zeros(u[e].shape, dtype=u.dtype)
        for l in range(d):
            Q = ref.Q[l]
            for m in range(d):
                g = G[:, l, m][:, None]
                if form == "skew":
                    r += 0.5 * (Q.T @ (g * f[m]) - g * (Q @ f[m]))
                else:
                    r += Q.T @ (g * f[m])
        for z in range(ref.Nf):
            e2, z2 = geo.nbr_elem[e, z], geo.nbr_face[e, z]
            ext = uf[z2][e2][geo.perm[e, z]]
            n = geo.n_fac[z][e]
            fstar = model.numflux(uf[z][e], ext, n)
            BJ = (ref.wf[z] * geo.Jf[z][e])[:, None]
            if form == "skew":
                fn = sum(n[:, m, None] * (ref.R[z] @ f[m]) for m in range(d))
                r -= ref.R[z].T @ (BJ * (fstar - 0.5 * fn))
            else:
                r -= ref.R[z].T @ (BJ * fstar)
        out.append(r)
    return np.stack(out)


def rhs(D, um, model, form="skew", elems=None):
    """d u~/dt of Eq. (modal) with the weight-adjusted inverse (M = I): [e, Nc, Np]."""
    elems = np.arange(D.E) if elems is None else np.asarray(elems)
    r = nodal_residual(D, um, model, form, elems)
    y = np.einsum("ij,eic->ejc", D.V, r)
    return np.transpose(D.minv(y, elems), (0, 2, 1))
