"""Section 7.1-7.2: compressible Euler equations, entropy, entropy variables,
logarithmic mean, Ranocha's entropy-conservative flux, Davis wave speed and the
local Lax-Friedrichs interface flux.  Oracle (test infrastructure only).

States are arrays [..., d+2] ordered (rho, rho v_1..rho v_d, E).  The
functions accept complex input (complex-step differentiation): comparisons
use real parts and |.| is continued analytically as sign(Re x) x.

Readings of the print:
* Eq. (ranocha_flux), energy component: the factor 1/2 multiplies v^- . v^+
  only, i.e.  f_E = rho_ln {{v_m}} (v^-.v^+/2 + 1/((gamma-1) {{rho/p}}_ln))
  + (p^- v_m^+ + p^+ v_m^-)/2; with the factor on both terms the flux is not
  consistent with f_m (Definition 5).
* Log mean: the paper defers its near-equal-argument branch to Ranocha et al.
  (Algorithms 2 and 3 there).  Written here from the identity
  ln(b/a) = 2 artanh(f), f = (b-a)/(b+a): with u = f^2,
  {{a}}_ln = (a+b) / (2 + 2u/3 + 2u^2/5 + 2u^3/7 + ...), used for u < 1e-4,
  where the truncation after four terms is below 1.2e-17 relative (FP64; more terms
  in extended precision); otherwise (b-a)/ln(b/a).

Every function works in the floating-point type of its arguments (FP64, complex128
for complex steps, or np.longdouble for the extended-precision evaluation).
"""
import numpy as np

GAMMA = 1.4
LOGMEAN_CUTOFF = 1.0e-4


def _abs(x):
    return np.where(np.real(x) >= 0, x, -x)


def _max(a, b):
    return np.where(np.real(a) >= np.real(b), a, b)


def primitive(U, gamma=GAMMA):
    rho = U[..., 0]
    v = U[..., 1:-1] / rho[..., None]
    p = (gamma - 1.0) * (U[..., -1] - 0.5 * rho * np.sum(v * v, axis=-1))
    return rho, v, p


def conservative(rho, v, p, gamma=GAMMA):
    E = p / (gamma - 1.0) + 0.5 * rho * np.sum(v * v, axis=-1)
    return np.concatenate([rho[..., None], rho[..., None] * v, E[..., None]], axis=-1)


def euler_flux(U, m, gamma=GAMMA):
    """f_m(U) of Eq. (euler)."""
    rho, v, p = primitive(U, gamma)
    d = v.shape[-1]
    out = np.empty(U.shape, dtype=np.result_type(U, float))
    out[..., 0] = rho * v[..., m]
    for k in range(d):
        out[..., 1 + k] = rho * v[..., k] * v[..., m] + (p if k == m else 0.0)
    out[..., -1] = v[..., m] * (U[..., -1] + p)
    return out


def euler_flux_dir(U, n, gamma=GAMMA):
    return sum(n[..., m, None] * euler_flux(U, m, gamma) for m in range(n.shape[-1]))


def entropy(U, gamma=GAMMA):
    """S(U) = -rho/(gamma-1) ln(p / rho^gamma), Eq. (euler_entropy)."""
    rho, v, p = primitive(U, gamma)
    return -rho / (gamma - 1.0) * np.log(p / rho ** gamma)


def entropy_flux(U, m, gamma=GAMMA):
    """F_m(U) = -rho v_m/(gamma-1) ln(p / rho^gamma), Eq. (euler_entropy)."""
    rho, v, p = primitive(U, gamma)
    return -rho * v[..., m] / (gamma - 1.0) * np.log(p / rho ** gamma)


def entropy_vars(U, gamma=GAMMA):
    """W(U) = grad_U S: ((gamma - s)/(gamma-1) - rho|v|^2/(2p), rho v/p, -rho/p), s = ln(p/rho^gamma)."""
    rho, v, p = primitive(U, gamma)
    s = np.log(p) - gamma * np.log(rho)
    w1 = (gamma - s) / (gamma - 1.0) - rho * np.sum(v * v, axis=-1) / (2.0 * p)
    return np.concatenate([w1[..., None], (rho / p)[..., None] * v, (-rho / p)[..., None]], axis=-1)


def cons_from_entropy(w, gamma=GAMMA):
    """The inverse map U(w) of W: with b = -w_last = rho/p and v = w_v / b,
    s = gamma - (gamma-1)(w_1 + b|v|^2/2),  rho = (b e^s)^(-1/(gamma-1)),  p = rho/b."""
    b = -w[..., -1]
    v = w[..., 1:-1] / b[..., None]
    s = gamma - (gamma - 1.0) * (w[..., 0] + 0.5 * b * np.sum(v * v, axis=-1))
    rho = np.exp(-(s + np.log(b)) / (gamma - 1.0))
    p = rho / b
    return conservative(rho, v, p, gamma)


def _artanh_series(u):
    """2 artanh(f)/f = 2 sum_k u^k/(2k+1), u = f^2, truncated for u < LOGMEAN_CUTOFF
    where the first omitted term is below the unit roundoff of the working precision:
    four terms in FP64 (truncation < 1.2e-17), more in extended precision."""
    R = np.real(np.asarray(u)).dtype.type
    eps = np.finfo(R).eps
    K = 3
    while LOGMEAN_CUTOFF ** (K + 1) / (2 * K + 3) > eps / 16:
        K += 1
    acc = R(2) / R(2 * K + 1)
    for k in range(K - 1, -1, -1):
        acc = R(2) / R(2 * k + 1) + u * acc
    return acc


def log_mean(a, b):
    """{{a}}_ln of Section 7.2 (series branch for nearly equal arguments)."""
    f = (b - a) / (b + a)
    u = f * f
    series = (a + b) / _artanh_series(u)
    safe_b = np.where(np.real(u) < LOGMEAN_CUTOFF, 2.0 * a + 1.0, b)   # avoid 0/0 in the unused branch
    direct = (safe_b - a) / np.log(safe_b / a)
    return np.where(np.real(u) < LOGMEAN_CUTOFF, series, direct)


def inv_log_mean(a, b):
    """1 / {{a}}_ln with the same branches."""
    f = (b - a) / (b + a)
    u = f * f
    series = _artanh_series(u) / (a + b)
    safe_b = np.where(np.real(u) < LOGMEAN_CUTOFF, 2.0 * a + 1.0, b)
    direct = np.log(safe_b / a) / (safe_b - a)
    return np.where(np.real(u) < LOGMEAN_CUTOFF, series, direct)


def ranocha_flux(UL, UR, m, gamma=GAMMA):
    """f_m^#(U^-, U^+) of Eq. (ranocha_flux) (energy term as read above)."""
    rL, vL, pL = primitive(UL, gamma)
    rR, vR, pR = primitive(UR, gamma)
    d = vL.shape[-1]
    rho_ln = log_mean(rL, rR)
    inv_beta_ln = inv_log_mean(rL / pL, rR / pR)
    vavg = 0.5 * (vL + vR)
    pavg = 0.5 * (pL + pR)
    f_rho = rho_ln * vavg[..., m]
    shape = np.broadcast(rL, rR).shape + (d + 2,)
    out = np.empty(shape, dtype=np.result_type(UL, UR, float))
    out[..., 0] = f_rho
    for k in range(d):
        out[..., 1 + k] = f_rho * vavg[..., k] + (pavg if k == m else 0.0)
    out[..., -1] = (f_rho * (0.5 * np.sum(vL * vR, axis=-1) + inv_beta_ln / (gamma - 1.0))
                    + 0.5 * (pL * vR[..., m] + pR * vL[..., m]))
    return out


def ranocha_flux_dir(UL, UR, n, gamma=GAMMA):
    """f^#(U^-, U^+, n) = sum_m n_m f_m^#(U^-, U^+)."""
    return sum(n[..., m, None] * ranocha_flux(UL, UR, m, gamma) for m in range(n.shape[-1]))


def sound_speed(U, gamma=GAMMA):
    rho, v, p = primitive(U, gamma)
    return np.sqrt(gamma * p / rho)


def davis_speed(UL, UR, n, gamma=GAMMA):
    """lambda(U^-, U^+, n) of Eq. (wave_speed)."""
    _, vL, _ = primitive(UL, gamma)
    _, vR, _ = primitive(UR, gamma)
    return (_max(_abs(np.sum(vL * n, axis=-1)), _abs(np.sum(vR * n, axis=-1)))
            + _max(sound_speed(UL, gamma), sound_speed(UR, gamma)))


def interface_flux(UL, UR, n, dissipation=True, gamma=GAMMA):
    """f^*(U^-, U^+, n) of Eq. (num_flux); without the dissipative term when dissipation is False."""
    f = ranocha_flux_dir(UL, UR, n, gamma)
    if dissipation:
        f = f - 0.5 * davis_speed(UL, UR, n, gamma)[..., None] * (UR - UL)
    return f
