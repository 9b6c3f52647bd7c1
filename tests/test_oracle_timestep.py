"""Pins of the RKF45 oracle (oracle/timestep.py) to facts independent of it:
consistency of the tableau (row sums = nodes, weights sum to 1), the
convergence orders 4 (propagated) and 5 (error estimate) on an ODE with a
closed-form solution, and a full adaptive run meeting its tolerance."""

import numpy as np

from oracle import timestep as ts


def test_tableau_consistency():
    for s in range(6):
        assert abs(sum(ts.A[s]) - ts.C[s]) < 1e-15
    assert abs(ts.B4.sum() - 1.0) < 1e-15 and abs(ts.B5.sum() - 1.0) < 1e-15


def _rhs(t, y):
    # y' = -y + sin t, y(0) = 1: y = (3 e^{-t} + sin t - cos t) / 2
    return -y + np.sin(t)


def _exact(t):
    return (3 * np.exp(-t) + np.sin(t) - np.cos(t)) / 2


def fixed_steps(n, which):
    y, t, dt = np.array([1.0]), 0.0, 1.0 / n
    for _ in range(n):
        y4, y5 = ts.rkf45_step(_rhs, t, y, dt)
        y, t = (y4 if which == 4 else y5), t + dt
    return abs(y[0] - _exact(1.0))


def test_orders_four_and_five():
    e4 = [fixed_steps(n, 4) for n in (8, 16, 32)]
    e5 = [fixed_steps(n, 5) for n in (8, 16, 32)]
    o4 = np.log2(e4[1] / e4[2])
    o5 = np.log2(e5[1] / e5[2])
    assert 3.7 < o4 < 4.4 and 4.6 < o5 < 5.5, (o4, o5)


def test_adaptive_run_meets_tolerance():
    y, dt, acc, rej = ts.integrate(_rhs, np.array([1.0]), 5.0, 0.5, 1e-8)
    assert abs(y[0] - _exact(5.0)) < 1e-6 and acc > 5
    # a first step far too large is rejected and shrunk
    _, _, acc2, rej2 = ts.integrate(lambda t, y: -50.0 * y, np.array([1.0]), 0.1, 0.1, 1e-6)
    assert rej2 >= 1 and acc2 >= 1
