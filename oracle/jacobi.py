"""Section 2.5: normalized Jacobi polynomials, Gauss-Jacobi quadrature, Lagrange polynomials.

Oracle (test infrastructure only).

Every routine works in the floating-point type of its arguments (or the ``dtype``
given): FP64 by default, ``np.longdouble`` for the extended-precision evaluation of
the residual (oracle/extended.py).
"""
from fractions import Fraction
from math import factorial

import numpy as np


def _real_type(dtype):
    return np.dtype(dtype).type


def _working_type(*arrays):
    """The float type of the arguments (FP64 for integers and Python floats)."""
    t = np.result_type(*[np.asarray(a) for a in arrays], np.float64)
    return t.type


def _recurrence(n, a, b, dtype=float):
    """Monic recurrence p_{k+1} = (x - alpha_k) p_k - beta_k p_{k-1} for the weight
    (1-x)^a (1+x)^b on [-1,1]; returns alpha_0..alpha_{n-1}, beta_0..beta_{n-1}
    with beta_0 = integral of the weight = 2^(a+b+1) a! b! / (a+b+1)!.

    The parameters used by the method are integers, so every coefficient is a
    rational number: it is formed exactly and rounded once to ``dtype``."""
    a, b = int(a), int(b)
    T = _real_type(dtype)
    rat = lambda f: T(f.numerator) / T(f.denominator)
    alpha = np.zeros(n, dtype=T)
    beta = np.zeros(n, dtype=T)
    for k in range(n):
        s = 2 * k + a + b
        if k == 0:
            alpha[k] = rat(Fraction(b - a, a + b + 2))
            beta[k] = rat(Fraction(2 ** (a + b + 1) * factorial(a) * factorial(b), factorial(a + b + 1)))
        else:
            alpha[k] = rat(Fraction(b * b - a * a, s * (s + 2)))
            beta[k] = rat(Fraction(4 * k * (k + a) * (k + b) * (k + a + b), s * s * (s + 1) * (s - 1)))
    return alpha, beta


def jacobi_p(n, a, b, x):
    """Values of the normalized Jacobi polynomials P_0..P_n^{(a,b)} at x: shape [n+1, len(x)].

    Normalized so that int P_i P_j (1-x)^a (1+x)^b dx = delta_ij (Section 2.5),
    built with the orthonormal form of the three-term recurrence.
    """
    T = _working_type(x)
    x = np.asarray(x, dtype=T)
    alpha, beta = _recurrence(n + 1, a, b, T)
    sb = np.sqrt(beta)
    P = np.zeros((n + 1,) + x.shape, dtype=T)
    P[0] = 1 / sb[0]
    if n >= 1:
        P[1] = (x - alpha[0]) * P[0] / sb[1]
    for k in range(1, n):
        P[k + 1] = ((x - alpha[k]) * P[k] - sb[k] * P[k - 1]) / sb[k + 1]
    return P


def _jacobi_p_deriv(n, a, b, x):
    """(P_n, dP_n/dx) of the normalized polynomial, by differentiating the recurrence."""
    T = x.dtype.type
    alpha, beta = _recurrence(n + 1, a, b, T)
    sb = np.sqrt(beta)
    p0, d0 = np.full(x.shape, 1 / sb[0], dtype=T), np.zeros(x.shape, dtype=T)
    if n == 0:
        return p0, d0
    p1, d1 = (x - alpha[0]) * p0 / sb[1], p0 / sb[1]
    for k in range(1, n):
        p2 = ((x - alpha[k]) * p1 - sb[k] * p0) / sb[k + 1]
        d2 = ((x - alpha[k]) * d1 + p1 - sb[k] * d0) / sb[k + 1]
        p0, d0, p1, d1 = p1, d1, p2, d2
    return p1, d1


def gauss_jacobi(q, a, b, dtype=float):
    """Gauss rule with q+1 nodes for the weight (1-x)^a (1+x)^b (Section 2.5).

    Nodes are the roots of P_{q+1}^{(a,b)}, i.e. the eigenvalues of the
    symmetric tridiagonal Jacobi matrix; weights are beta_0 times the squared
    first components of the normalized eigenvectors (Golub-Welsch), in FP64.
    For a wider ``dtype`` the FP64 nodes are then polished by Newton's method on
    P_{q+1} in that type and the weights recomputed as Christoffel numbers,
    w_i = 1 / sum_{k<=q} P_k(x_i)^2 (orthonormal P_k).
    """
    n = q + 1
    alpha, beta = _recurrence(n, a, b)
    Tm = np.diag(alpha) + np.diag(np.sqrt(beta[1:]), 1) + np.diag(np.sqrt(beta[1:]), -1)
    x, V = np.linalg.eigh(Tm)
    w = beta[0] * V[0, :] ** 2
    T = _real_type(dtype)
    if np.finfo(T).eps >= np.finfo(np.float64).eps:
        return x, w
    x = x.astype(T)
    for _ in range(8):
        p, dp = _jacobi_p_deriv(n, a, b, x)
        step = p / dp
        x = x - step
        if np.all(np.abs(step) <= 4 * np.finfo(T).eps):
            break
    P = jacobi_p(q, a, b, x)
    w = 1 / np.sum(P * P, axis=0)
    return x, w


def lagrange(nodes, x):
    """L[i, t] = ell_i(x_t), the Lagrange polynomials of Eq. (lagrange)."""
    T = _working_type(nodes, x)
    nodes = np.asarray(nodes, dtype=T)
    x = np.atleast_1d(np.asarray(x, dtype=T))
    n = len(nodes)
    L = np.ones((n, len(x)), dtype=T)
    for i in range(n):
        for j in range(n):
            if j != i:
                L[i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return L


def lagrange_deriv(nodes, x):
    """dL[i, t] = d ell_i / d eta at x_t, by the product rule applied to Eq. (lagrange)."""
    T = _working_type(nodes, x)
    nodes = np.asarray(nodes, dtype=T)
    x = np.atleast_1d(np.asarray(x, dtype=T))
    n = len(nodes)
    dL = np.zeros((n, len(x)), dtype=T)
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.ones(len(x), dtype=T) / (nodes[i] - nodes[k])
            for j in range(n):
                if j != i and j != k:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            dL[i] += term
    return dL
