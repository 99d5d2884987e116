"""Classical four-stage Runge-Kutta step (the paper integrates with an
eighth-order Dormand-Prince method; the library steps with RK4).
Oracle (test infrastructure only)."""


def rk4_step(f, u, dt):
    k1 = f(u)
    k2 = f(u + 0.5 * dt * k1)
    k3 = f(u + 0.5 * dt * k2)
    k4 = f(u + dt * k3)
    return u + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
