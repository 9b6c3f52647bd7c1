"""Pins of the RKF45 oracle (oracle/timestep.py) to facts independent of it:
consistency of the tableau (row sums = nodes, weights sum to 1), Butcher's
order conditions for all rooted trees up to five nodes (exactly order 4 for
the propagated weights, 5 for the estimator), the convergence orders 4 and 5
on a linear ODE and on a nonlinear non-autonomous system with closed-form
solutions, and a full adaptive run meeting its tolerance."""

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


def _order_conditions(A, b, c):
    """Butcher's order conditions sum_i b_i Phi_i(t) = 1/gamma(t) for every
    rooted tree t with up to five nodes (1 + 1 + 2 + 4 + 9 = 17 trees), as
    (order, residual) pairs; c_i = sum_j a_ij."""
    n = len(b)
    a = np.zeros((n, n))
    for i, row in enumerate(A):
        a[i, :len(row)] = row
    ac, ac2, ac3 = a @ c, a @ c**2, a @ c**3
    aac = a @ ac
    conds = [
        (1, b.sum(), 1),
        (2, b @ c, 1 / 2),
        (3, b @ c**2, 1 / 3), (3, b @ ac, 1 / 6),
        (4, b @ c**3, 1 / 4), (4, b @ (c * ac), 1 / 8), (4, b @ ac2, 1 / 12), (4, b @ aac, 1 / 24),
        (5, b @ c**4, 1 / 5), (5, b @ (c**2 * ac), 1 / 10), (5, b @ (c * ac2), 1 / 15),
        (5, b @ (c * aac), 1 / 30), (5, b @ ac**2, 1 / 20), (5, b @ ac3, 1 / 20),
        (5, b @ (a @ (c * ac)), 1 / 40), (5, b @ (a @ ac2), 1 / 60), (5, b @ (a @ aac), 1 / 120),
    ]
    return [(p, lhs - rhs) for p, lhs, rhs in conds]


def _order(A, b, c):
    """Largest p such that every condition of order <= p holds to 1e-14."""
    p = 0
    for q in range(1, 6):
        if all(abs(r) < 1e-14 for o, r in _order_conditions(A, b, c) if o == q):
            p = q
        else:
            break
    return p


def test_tableau_satisfies_butcher_order_conditions():
    # the propagated weights are exactly fourth order, the estimator's fifth
    assert _order(ts.A, ts.B4, ts.C) == 4
    assert _order(ts.A, ts.B5, ts.C) == 5
    # a mistake that keeps the row sums (two entries of a row swapped) is caught
    bad = [list(r) for r in ts.A]
    bad[4][1], bad[4][2] = bad[4][2], bad[4][1]
    assert abs(sum(bad[4]) - ts.C[4]) < 1e-15
    assert _order(bad, ts.B5, ts.C) < 5 and _order(bad, ts.B4, ts.C) < 4


def test_orders_on_a_nonlinear_system():
    # x' = -r y, y' = r x with r = x^2 + y^2 (conserved): rotation at rate r,
    # plus the non-autonomous z' = -2 t z^2, z(0) = 1: z = 1 / (1 + t^2)
    def rhs(t, u):
        r = u[0] ** 2 + u[1] ** 2
        return np.array([-r * u[1], r * u[0], -2.0 * t * u[2] ** 2])

    u0 = np.array([0.6, 0.8, 1.0])  # r = 1

    def err(n, which):
        u, t, dt = u0.copy(), 0.0, 2.0 / n
        for _ in range(n):
            y4, y5 = ts.rkf45_step(rhs, t, u, dt)
            u, t = (y4 if which == 4 else y5), t + dt
        ex = np.array([0.6 * np.cos(2.0) - 0.8 * np.sin(2.0), 0.6 * np.sin(2.0) + 0.8 * np.cos(2.0),
                       1.0 / 5.0])
        return np.abs(u - ex).max()

    e4 = [err(n, 4) for n in (16, 32, 64)]
    e5 = [err(n, 5) for n in (16, 32, 64)]
    o4, o5 = np.log2(e4[1] / e4[2]), np.log2(e5[1] / e5[2])
    assert 3.7 < o4 < 4.4 and 4.6 < o5 < 5.6, (o4, o5)
