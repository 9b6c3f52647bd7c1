"""Pins that tie the oracle to facts fixed by the paper and by Stokes theory.

Each pin takes an `oracle.Oracle` so the same battery also runs against
deliberately broken copies of the oracle (tests/test_oracle_mutations.py).

Facts used (none of them is the oracle's own formula typed again):
  * r -> 0 limits of s1/r and s2/r^3 (Sec. 3.4, printed after s1, s2);
  * far field: for r >> delta the regularized sum is the Stokeslet sum with
    G = (I/r + r r^T / r^3) / (8 pi mu) (Sec. 2.2, below Eq. bi2);
  * a sphere of radius a under uniform traction f0 moves rigidly with
    U = F / (6 pi mu a), F = 4 pi a^2 f0, i.e. S[f0] = 2 a f0 / (3 mu);
  * S[n] = 0 on any closed surface (the Stokeslet is divergence-free);
  * double layer of a constant density q: q inside, 0 outside, q/2 on the
    surface (Gauss-type identity of the stresslet);
  * regularization error O(delta^5) (Sec. 3.4, after the limits) and
    fourth-order convergence in h with delta proportional to h (Sec. 3.6,
    "Accuracy and work complexity").
"""

from __future__ import annotations

import math

import numpy as np

import capsule_inputs as ci


def sphere_axisym_quadrature(a: float, delta: float, n_near: int = 200, n_far: int = 400,
                             K: int = 256):
    """Nodes and weights on a sphere of radius a, fine near the north pole.

    Gauss-Legendre in the polar angle on [0, 12 delta / a] and on the rest,
    trapezoid in the azimuth: a quadrature of the continuous surface integral
    accurate far beyond the regularization error for a target at (0, 0, a).
    """
    t1 = min(12.0 * delta / a, math.pi / 2)
    xs, ws = np.polynomial.legendre.leggauss(n_near)
    th1, w1 = 0.5 * t1 * (xs + 1), 0.5 * t1 * ws
    xs2, ws2 = np.polynomial.legendre.leggauss(n_far)
    th2, w2 = t1 + 0.5 * (math.pi - t1) * (xs2 + 1), 0.5 * (math.pi - t1) * ws2
    th = np.concatenate([th1, th2])
    wt = np.concatenate([w1, w2])
    ph = 2 * math.pi * np.arange(K) / K
    T, P = np.meshgrid(th, ph, indexing="ij")
    X = a * np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    W = (a * a * np.sin(T) * wt[:, None] * (2 * math.pi / K)).ravel()
    return X, W


# ----------------------------------------------------------------- single layer

def pin_sl_self_limit(orc):
    """One node at the target: u = w f s1/r|_{r=0} / (8 pi mu) (Sec. 3.4 limit)."""
    for delta, mu in ((0.1, 1.0), (0.37, 2.5)):
        f = np.array([[0.3, -1.2, 2.0]])
        u = orc.sl([[1.0, 2.0, 3.0]], [0.7], f, [[1.0, 2.0, 3.0]], delta, mu)
        lim = 16.0 / (3.0 * delta * math.sqrt(math.pi))
        assert np.allclose(u, 0.7 * f * lim / (8 * math.pi * mu), rtol=1e-14, atol=0)


def pin_sl_far_field_is_stokeslet(orc):
    rng = np.random.default_rng(11)
    X = rng.standard_normal((40, 3))
    Y = rng.standard_normal((7, 3)) + 20.0
    w = rng.uniform(0.1, 1.0, 40)
    f = rng.standard_normal((40, 3))
    mu = 1.7
    u = orc.sl(X, w, f, Y, 0.5, mu)  # r / delta > 30: s1 = s2 = 1 to rounding
    ref = np.zeros((7, 3))
    for t in range(7):
        for j in range(40):
            r = Y[t] - X[j]
            rn = np.linalg.norm(r)
            G = (np.eye(3) / rn + np.outer(r, r) / rn ** 3) / (8 * math.pi * mu)
            ref[t] += w[j] * G @ f[j]
    assert np.allclose(u, ref, rtol=1e-13, atol=0)


def pin_sl_sphere_uniform_traction(orc):
    """S[f0] = 2 a f0 / (3 mu) on a sphere (rigid translation), any direction."""
    for a, mu, delta in ((1.0, 1.0, 0.2), (0.7, 2.0, 0.1)):
        X, W = sphere_axisym_quadrature(a, delta)
        for f0 in (np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, -2.0]),
                   np.array([0.3, 0.4, 0.5])):
            u = orc.sl(X, W, np.broadcast_to(f0, X.shape), [[0.0, 0.0, a]], delta, mu)
            assert np.allclose(u[0], 2 * a * f0 / (3 * mu), rtol=0, atol=1e-12)


def pin_sl_normal_density_vanishes(orc):
    for delta in (0.3, 0.1):
        X, W = sphere_axisym_quadrature(1.0, delta)
        u = orc.sl(X, W, X, [[0.0, 0.0, 1.0]], delta, 1.0)
        assert np.abs(u).max() < 1e-12


def pin_sl_delta_fifth_order(orc):
    """Regularization error ~ delta^5: successive differences shrink by ~32."""
    vals = []
    for delta in (0.1, 0.05, 0.025):
        X, W = sphere_axisym_quadrature(1.0, delta, n_near=300, n_far=600, K=64)
        u = orc.sl(X, W, X ** 2, [[0.0, 0.0, 1.0]], delta, 1.0)
        vals.append(u[0])
    d1 = np.abs(vals[1] - vals[0]).max()
    d2 = np.abs(vals[2] - vals[1]).max()
    assert 25.0 < d1 / d2 < 40.0, d1 / d2


def pin_sl_h_order_on_patches(orc):
    """Ellipsoid, delta = 2h: S[n] -> 0 at fourth order or better in h."""
    rng = np.random.default_rng(7)
    errs = []
    for m in (33, 65, 129):
        s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), m)
        idx = rng.choice(s.N, 48, replace=False)
        errs.append(np.abs(orc.sl(s.X, s.w, s.n, s.X[idx], 2 * s.h, 1.0)).max())
    assert errs[-1] < 1e-5
    assert errs[1] / errs[2] > (128.0 / 64.0) ** 4, errs


def pin_sl_per_target_delta(orc):
    """delta belongs to the target (Eq. regparam): array == per-target scalars."""
    s = ci.make_surface(ci.Sphere(1.0), 9)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((s.N, 3))
    Y = s.X[:5]
    deltas = np.array([0.2, 0.35, 0.5, 0.9, 1.3])
    u = orc.sl(s.X, s.w, f, Y, deltas, 1.0)
    for t in range(5):
        ut = orc.sl(s.X, s.w, f, Y[t:t + 1], deltas[t], 1.0)
        assert np.array_equal(u[t], ut[0])


def pin_sl_mu_scaling_and_linearity(orc):
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 7)
    rng = np.random.default_rng(4)
    f1, f2 = rng.standard_normal((2, s.N, 3))
    u1 = orc.sl(s.X, s.w, f1, s.X, 0.4, 1.0)
    u2 = orc.sl(s.X, s.w, f2, s.X, 0.4, 1.0)
    u12 = orc.sl(s.X, s.w, f1 + 2 * f2, s.X, 0.4, 1.0)
    assert np.allclose(u12, u1 + 2 * u2, rtol=1e-12, atol=1e-14)
    assert np.allclose(orc.sl(s.X, s.w, f1, s.X, 0.4, 4.0), u1 / 4.0, rtol=1e-14, atol=0)


def pin_sl_rotation_translation_covariance(orc):
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 7)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((s.N, 3))
    Q = ci.random_rotation(rng)
    shift = np.array([3.0, -1.0, 0.5])
    u = orc.sl(s.X, s.w, f, s.X, 0.4, 1.0)
    ur = orc.sl(s.X @ Q.T + shift, s.w, f @ Q.T, s.X @ Q.T + shift, 0.4, 1.0)
    assert np.allclose(ur, u @ Q.T, rtol=1e-10, atol=1e-13)


SL_PINS = [pin_sl_self_limit, pin_sl_far_field_is_stokeslet, pin_sl_sphere_uniform_traction,
           pin_sl_normal_density_vanishes, pin_sl_delta_fifth_order, pin_sl_h_order_on_patches,
           pin_sl_per_target_delta, pin_sl_mu_scaling_and_linearity,
           pin_sl_rotation_translation_covariance]


# ----------------------------------------------------------------- double layer

def pin_dl_constant_density_sphere(orc):
    """Constant q: D = q/2 on the surface (exact on the sphere for small delta)."""
    for a, delta in ((1.0, 0.2), (0.6, 0.05)):
        X, W = sphere_axisym_quadrature(a, delta)
        for q0 in (np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0]),
                   np.array([0.2, -0.7, 0.4])):
            u = orc.dl(X, W, X / a, np.broadcast_to(q0, X.shape), [[0.0, 0.0, a]], delta)
            assert np.allclose(u[0], q0 / 2, rtol=0, atol=1e-12)


def pin_dl_constant_density_inside_outside(orc):
    # targets 0.35+ away from the surface: the integrand is smooth, so the POU
    # trapezoid rule converges super-algebraically (m = 129: ~5e-11)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 129)
    q0 = np.array([0.3, -0.5, 0.8])
    q = np.broadcast_to(q0, s.X.shape)
    Y = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.1], [3.0, 0.0, 0.0], [0.0, -2.0, 1.0]])
    u = orc.dl(s.X, s.w, s.n, q, Y, 2 * s.h)
    assert np.allclose(u[:2], q0, rtol=0, atol=1e-9)
    assert np.allclose(u[2:], 0.0, rtol=0, atol=1e-9)


def pin_dl_constant_density_on_patches(orc):
    rng = np.random.default_rng(8)
    q0 = np.array([0.0, 1.0, 0.0])
    errs = []
    for m in (65, 129):
        s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), m)
        idx = rng.choice(s.N, 32, replace=False)
        u = orc.dl(s.X, s.w, s.n, np.broadcast_to(q0, s.X.shape), s.X[idx], 2 * s.h)
        errs.append(np.abs(u - q0 / 2).max())
    # fourth order or better in h with delta = 2h (measured ratio ~29)
    assert errs[-1] < 1e-4 and errs[0] / errs[1] > 16.0, errs


def pin_dl_delta_fifth_order(orc):
    vals = []
    for delta in (0.1, 0.05, 0.025):
        X, W = sphere_axisym_quadrature(1.0, delta, n_near=300, n_far=600, K=64)
        q = np.zeros_like(X)
        q[:, 2] = X[:, 2] ** 2
        vals.append(orc.dl(X, W, X, q, [[0.0, 0.0, 1.0]], delta)[0])
    d1 = np.abs(vals[1] - vals[0]).max()
    d2 = np.abs(vals[2] - vals[1]).max()
    assert 25.0 < d1 / d2 < 40.0, d1 / d2


def pin_dl_self_term_zero_and_far_field(orc):
    u = orc.dl([[1.0, 1.0, 1.0]], [1.0], [[0.0, 0.0, 1.0]], [[1.0, 2.0, 3.0]],
               [[1.0, 1.0, 1.0]], 0.2)
    assert np.all(u == 0.0)
    rng = np.random.default_rng(12)
    X = rng.standard_normal((30, 3))
    n = rng.standard_normal((30, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    q = rng.standard_normal((30, 3))
    w = rng.uniform(0.1, 1, 30)
    Y = rng.standard_normal((5, 3)) + 15.0
    u = orc.dl(X, w, n, q, Y, 0.3)
    ref = np.zeros((5, 3))
    for t in range(5):
        for j in range(30):
            d = Y[t] - X[j]
            r = np.linalg.norm(d)
            ref[t] += w[j] * (-6.0) * (d @ q[j]) * (d @ n[j]) * d / r ** 5 / (8 * math.pi)
    assert np.allclose(u, ref, rtol=1e-13, atol=0)


DL_PINS = [pin_dl_constant_density_sphere, pin_dl_constant_density_inside_outside,
           pin_dl_constant_density_on_patches, pin_dl_delta_fifth_order,
           pin_dl_self_term_zero_and_far_field]
