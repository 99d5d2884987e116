"""Analytic initial conditions (Section 7.4, 7.5) and seeded perturbations.

All functions take physical points ``x`` of shape [..., d] and return the
conservative state [..., d+2] ordered (rho, rho v_1..rho v_d, E) as in the
Euler system of Section 7.1.
"""
import numpy as np


def conservative_from_primitive(rho, vel, p, gamma=1.4):
    """(rho, v, p) -> (rho, rho v, p/(gamma-1) + rho |v|^2 / 2)."""
    vel = np.asarray(vel)
    E = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return np.concatenate([rho[..., None], rho[..., None] * vel, E[..., None]], axis=-1)


def isentropic_vortex(x, center, L, strength=5.0, gamma=1.4, background=(1.0, 1.0, 1.0, 1.0)):
    """Shu's isentropic vortex on a background (rho, u, v, p) = (1, 1, 1, 1).

    Distances are measured in units of L/10, so the vortex occupies the same
    fraction of the domain for any L.
    """
    rho0, u0, v0, p0 = background
    xb = (x[..., 0] - center[0]) * 10.0 / L
    yb = (x[..., 1] - center[1]) * 10.0 / L
    r2 = xb * xb + yb * yb
    g = strength / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    T = p0 / rho0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = rho0 * (T / (p0 / rho0)) ** (1.0 / (gamma - 1.0))
    p = p0 * (rho / rho0) ** gamma
    vel = np.stack([u0 - g * yb, v0 + g * xb], axis=-1)
    return conservative_from_primitive(rho, vel, p, gamma)


def taylor_green(x, mach=0.1, gamma=1.4):
    """Taylor-Green vortex of Section 7.5 (rho = 1, w = 0).

    The pressure uses the symmetric form 1/(gamma Ma^2) + (2 cos 2x1 + 2 cos 2x2
    + cos 2x1 cos 2x3 + cos 2x2 cos 2x3)/16: the printed coefficient of cos 2x1
    (1 instead of 2) breaks the x1 <-> x2 symmetry of the velocity field.
    """
    x1, x2, x3 = x[..., 0], x[..., 1], x[..., 2]
    rho = np.ones_like(x1)
    vel = np.stack([np.sin(x1) * np.cos(x2) * np.cos(x3),
                    -np.cos(x1) * np.sin(x2) * np.cos(x3),
                    np.zeros_like(x1)], axis=-1)
    p = 1.0 / (gamma * mach ** 2) + (2 * np.cos(2 * x1) + 2 * np.cos(2 * x2)
                                     + np.cos(2 * x1) * np.cos(2 * x3)
                                     + np.cos(2 * x2) * np.cos(2 * x3)) / 16.0
    return conservative_from_primitive(rho, vel, p, gamma)


def density_wave(x, L=2.0, gamma=1.4):
    """Smooth density wave of Section 7.4: rho = 1 + sin(2 pi sum(x)/L)/5, v = 1, p = 1."""
    d = x.shape[-1]
    rho = 1.0 + 0.2 * np.sin(2 * np.pi / L * np.sum(x, axis=-1))
    vel = np.ones(x.shape[:-1] + (d,))
    p = np.ones_like(rho)
    return conservative_from_primitive(rho, vel, p, gamma)


def seeded_uniform(seed, shape, lo, hi):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def seeded_normal(seed, shape, scale):
    return np.random.default_rng(seed).normal(0.0, scale, size=shape)


def max_wave_speed_sampled(state_fn, dim, L, n=64, gamma=1.4):
    """max(|v| + c) of an analytic state sampled on an n^d grid (used to fix dt)."""
    g = (np.arange(n) + 0.5) * L / n
    pts = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), axis=-1).reshape(-1, dim)
    U = state_fn(pts)
    rho = U[:, 0]
    v = U[:, 1:1 + dim] / rho[:, None]
    p = (gamma - 1.0) * (U[:, -1] - 0.5 * rho * np.sum(v * v, axis=1))
    return float(np.max(np.linalg.norm(v, axis=1) + np.sqrt(gamma * p / rho)))
