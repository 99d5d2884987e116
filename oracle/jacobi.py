"""Section 2.5: normalized Jacobi polynomials, Gauss-Jacobi quadrature, Lagrange polynomials.

Oracle (test infrastructure only).
"""
from math import lgamma, exp, sqrt
import numpy as np


def _recurrence(n, a, b):
    """Monic recurrence p_{k+1} = (x - alpha_k) p_k - beta_k p_{k-1} for the weight
    (1-x)^a (1+x)^b on [-1,1]; returns alpha_0..alpha_{n-1}, beta_0..beta_{n-1}
    with beta_0 = integral of the weight."""
    alpha = np.zeros(n)
    beta = np.zeros(n)
    for k in range(n):
        s = 2 * k + a + b
        if k == 0:
            alpha[k] = (b - a) / (a + b + 2.0)
            beta[k] = exp((a + b + 1) * np.log(2.0) + lgamma(a + 1) + lgamma(b + 1) - lgamma(a + b + 2))
        else:
            alpha[k] = (b * b - a * a) / (s * (s + 2.0))
            beta[k] = 4.0 * k * (k + a) * (k + b) * (k + a + b) / (s * s * (s + 1.0) * (s - 1.0))
    return alpha, beta


def jacobi_p(n, a, b, x):
    """Values of the normalized Jacobi polynomials P_0..P_n^{(a,b)} at x: shape [n+1, len(x)].

    Normalized so that int P_i P_j (1-x)^a (1+x)^b dx = delta_ij (Section 2.5),
    built with the orthonormal form of the three-term recurrence.
    """
    x = np.asarray(x, dtype=float)
    alpha, beta = _recurrence(n + 1, a, b)
    P = np.zeros((n + 1,) + x.shape)
    P[0] = 1.0 / sqrt(beta[0])
    if n >= 1:
        P[1] = (x - alpha[0]) * P[0] / sqrt(beta[1])
    for k in range(1, n):
        P[k + 1] = ((x - alpha[k]) * P[k] - sqrt(beta[k]) * P[k - 1]) / sqrt(beta[k + 1])
    return P


def gauss_jacobi(q, a, b):
    """Gauss rule with q+1 nodes for the weight (1-x)^a (1+x)^b (Section 2.5).

    Nodes are the roots of P_{q+1}^{(a,b)}, i.e. the eigenvalues of the
    symmetric tridiagonal Jacobi matrix; weights are beta_0 times the squared
    first components of the normalized eigenvectors (Golub-Welsch).
    """
    n = q + 1
    alpha, beta = _recurrence(n, a, b)
    T = np.diag(alpha) + np.diag(np.sqrt(beta[1:]), 1) + np.diag(np.sqrt(beta[1:]), -1)
    x, V = np.linalg.eigh(T)
    w = beta[0] * V[0, :] ** 2
    return x, w


def lagrange(nodes, x):
    """L[i, t] = ell_i(x_t), the Lagrange polynomials of Eq. (lagrange)."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    L = np.ones((n, len(x)))
    for i in range(n):
        for j in range(n):
            if j != i:
                L[i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return L


def lagrange_deriv(nodes, x):
    """dL[i, t] = d ell_i / d eta at x_t, by the product rule applied to Eq. (lagrange)."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    dL = np.zeros((n, len(x)))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.ones(len(x)) / (nodes[i] - nodes[k])
            for j in range(n):
                if j != i and j != k:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            dL[i] += term
    return dL
