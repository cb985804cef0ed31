"""The paper's hyperchaotic test system (Sec. 5, the 4D Lorenz-type example), for checking the
GPU generator of its data (test infrastructure only, like the rest of the oracle).

    dx/dt = a (y - x),  dy/dt = c x - y - x z + w,  dz/dt = -b z + x y,
    dw/dt = (c - 1) y + w - x^3 / b          (the paper's a = 15, b = 2, c = 28)

integrated with the classical fourth-order Runge-Kutta scheme at a fixed step (the paper
used an adaptive solver and does not state its steps; the step is an input here).
"""
import numpy as np


def lorenz4d_rhs(u, a=15.0, b=2.0, c=28.0):
    """Right-hand side for states u = (x, y, z, w) stacked on axis 0."""
    x, y, z, w = u
    return np.stack([a * (y - x), c * x - y - x * z + w, -b * z + x * y,
                     (c - 1.0) * y + w - x ** 3 / b])


def rk4_step(f, u, h):
    """One classical Runge-Kutta step of u' = f(u) with step h."""
    k1 = f(u)
    k2 = f(u + 0.5 * h * k1)
    k3 = f(u + 0.5 * h * k2)
    k4 = f(u + h * k3)
    return u + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def lorenz4d_snapshots(u0, steps, dt, a=15.0, b=2.0, c=28.0):
    """The (4, steps, cols) quaternion matrix whose entry (t, j) is the state x + y i + z j + w k
    of trajectory j after t + 1 steps; u0 is (4, cols)."""
    f = lambda u: lorenz4d_rhs(u, a, b, c)
    u = np.array(u0, dtype=np.float64)
    out = np.empty((4, steps, u.shape[1]))
    for t in range(steps):
        u = rk4_step(f, u, dt)
        out[:, t, :] = u
    return out
