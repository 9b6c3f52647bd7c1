"""Runge-Kutta-Fehlberg 4(5) adaptive time stepping, written out plainly.

Test infrastructure (see oracle/__init__.py): only tests, the smoke check and
the bench's baseline use it. Sec. 3.6 of arXiv 2310.13908 integrates
dx/dt = u_inf(x) + S[f](x) (Eq. bi_combined) with the explicit
Runge-Kutta-Fehlberg 4(5) scheme (Fehlberg 1969), fourth order in time, with a
fixed relative tolerance. The paper prints neither the tableau nor the step
controller; the tableau below is Fehlberg's published one, and these are the
readings for the rest:
  * the fourth-order solution is propagated (the scheme is "fourth-order
    accurate in time"), the fifth-order one only estimates the error;
  * error = max |y5 - y4| / max |y4| (relative, infinity norm), a step is
    accepted when error <= tol;
  * next dt = dt * min(5, max(0.2, 0.9 (tol / error)^(1/5))), also after a
    rejection; the last step is shortened to land on t_end.
"""

from __future__ import annotations

import numpy as np

# Fehlberg's RK4(5) tableau
C = np.array([0.0, 1 / 4, 3 / 8, 12 / 13, 1.0, 1 / 2])
A = [
    [],
    [1 / 4],
    [3 / 32, 9 / 32],
    [1932 / 2197, -7200 / 2197, 7296 / 2197],
    [439 / 216, -8.0, 3680 / 513, -845 / 4104],
    [-8 / 27, 2.0, -3544 / 2565, 1859 / 4104, -11 / 40],
]
B4 = np.array([25 / 216, 0.0, 1408 / 2565, 2197 / 4104, -1 / 5, 0.0])
B5 = np.array([16 / 135, 0.0, 6656 / 12825, 28561 / 56430, -9 / 50, 2 / 55])


def rkf45_step(rhs, t: float, y: np.ndarray, dt: float):
    """One Fehlberg step: returns (y4, y5)."""
    k = []
    for s in range(6):
        ys = y.copy()
        for j, a in enumerate(A[s]):
            ys = ys + dt * a * k[j]
        k.append(rhs(t + C[s] * dt, ys))
    y4 = y + dt * sum(b * kk for b, kk in zip(B4, k))
    y5 = y + dt * sum(b * kk for b, kk in zip(B5, k))
    return y4, y5


def step_error(y4: np.ndarray, y5: np.ndarray) -> float:
    return float(np.max(np.abs(y5 - y4)) / max(np.max(np.abs(y4)), 1e-300))


def next_dt(dt: float, err: float, tol: float) -> float:
    if err == 0.0:
        return dt * 5.0
    return dt * min(5.0, max(0.2, 0.9 * (tol / err) ** 0.2))


def integrate(rhs, y0: np.ndarray, t_end: float, dt0: float, tol: float, max_steps: int = 100000):
    """Adaptive RKF45 from t = 0 to t_end; returns (y, dt_next, accepted, rejected)."""
    t, y, dt = 0.0, np.array(y0, dtype=np.float64), float(dt0)
    acc = rej = 0
    while t < t_end and acc + rej < max_steps:
        h = min(dt, t_end - t)
        y4, y5 = rkf45_step(rhs, t, y, h)
        err = step_error(y4, y5)
        if err <= tol:
            t, y = t + h, y4
            acc += 1
        else:
            rej += 1
        dt = next_dt(h, err, tol)
    return y, dt, acc, rej
