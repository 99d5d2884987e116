"""Section 4.3: the normalized Proriol-Koornwinder-Dubiner basis (Eq. (principal_functions),
Eq. (modal_basis_2d), Eq. (modal_basis_3d)) and the generalized Vandermonde matrix
of Eq. (modal_to_nodal).  Oracle (test infrastructure only).

Modal multi-indices alpha in N(p) are ordered lexicographically with alpha_1
slowest (the order the C ABI documents).
"""
import numpy as np
from .jacobi import jacobi_p, _working_type


def modal_indices(dim, p):
    out = []
    for a1 in range(p + 1):
        for a2 in range(p + 1 - a1):
            if dim == 2:
                out.append((a1, a2))
            else:
                for a3 in range(p + 1 - a1 - a2):
                    out.append((a1, a2, a3))
    return np.array(out)


def pkd_eval(dim, p, eta):
    """phi_j(chi(eta)) for all modes j: shape [len(eta), N_p*]."""
    T = _working_type(eta)
    eta = np.atleast_2d(np.asarray(eta, dtype=T))
    idx = modal_indices(dim, p)
    out = np.zeros((eta.shape[0], len(idx)), dtype=T)
    sqrt2 = np.sqrt(T(2))
    for j, a in enumerate(idx):
        psi1 = sqrt2 * jacobi_p(a[0], 0, 0, eta[:, 0])[a[0]]
        psi2 = (1 - eta[:, 1]) ** a[0] * jacobi_p(a[1], 2 * a[0] + 1, 0, eta[:, 1])[a[1]]
        val = psi1 * psi2
        if dim == 3:
            psi3 = 2 * (1 - eta[:, 2]) ** (a[0] + a[1]) * jacobi_p(a[2], 2 * a[0] + 2 * a[1] + 2, 0, eta[:, 2])[a[2]]
            val = val * psi3
        out[:, j] = val
    return out


def vandermonde(ref, p):
    """V_ij = phi_j(xi_i) at the volume quadrature nodes of ``ref``."""
    return pkd_eval(ref.dim, p, ref.eta)
