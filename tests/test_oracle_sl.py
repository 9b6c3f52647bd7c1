"""Oracle single layer: pinned to closed forms, invariants and rates."""

import math

import numpy as np
import pytest

import capsule_inputs as ci
import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.SL_PINS, ids=lambda p: p.__name__)
def test_sl_pin(pin):
    pin(oracle.default())


def test_sl_brute_force_tiny_high_precision():
    """m = 3 and 4 grids (N = 24, 54): oracle vs a 50-digit direct sum."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(21)
    for m, shape in ((3, ci.Sphere(1.0)), (4, ci.Ellipsoid(1.0, 0.8, 0.5))):
        s = ci.make_surface(shape, m)
        f = rng.standard_normal((s.N, 3))
        delta, mu = 1.5 * s.h, 1.3
        u = oracle.sl(s.X, s.w, f, s.X, delta, mu)
        sq = mp.sqrt(mp.pi)
        for t in range(s.N):
            acc = [mp.mpf(0)] * 3
            for j in range(s.N):
                if s.w[j] == 0:
                    continue
                d = [mp.mpf(s.X[t, c]) - mp.mpf(s.X[j, c]) for c in range(3)]
                r = mp.sqrt(sum(x * x for x in d))
                if r == 0:
                    a = mp.mpf(16) / (3 * delta * sq)
                    b = mp.mpf(0)
                else:
                    p = r / delta
                    e = mp.exp(-p * p) / sq
                    s1 = mp.erf(p) - mp.mpf(2) / 3 * p * (2 * p * p - 5) * e
                    s2 = mp.erf(p) - mp.mpf(2) / 3 * p * (4 * p ** 4 - 14 * p * p + 3) * e
                    a, b = s1 / r, s2 / r ** 3
                fd = sum(mp.mpf(f[j, c]) * d[c] for c in range(3))
                for c in range(3):
                    acc[c] += mp.mpf(s.w[j]) * (mp.mpf(f[j, c]) * a + fd * d[c] * b)
            ref = np.array([float(x / (8 * mp.pi * mu)) for x in acc])
            assert np.allclose(u[t], ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())


def test_sl_zero_weight_sources_add_nothing():
    s = ci.make_surface(ci.Sphere(1.0), 9)
    rng = np.random.default_rng(2)
    f = rng.standard_normal((s.N, 3))
    keep = s.w != 0
    assert keep.sum() < s.N
    u_all = oracle.sl(s.X, s.w, f, s.X, 0.5)
    u_kept = oracle.sl(s.X[keep], s.w[keep], f[keep], s.X, 0.5)
    assert np.array_equal(u_all, u_kept)


def test_sl_empty_inputs_and_validation():
    assert oracle.sl(np.zeros((0, 3)), [], np.zeros((0, 3)), [[0, 0, 0]], 0.1).tolist() == [[0, 0, 0]]
    assert oracle.sl([[0, 0, 0]], [1.0], [[1, 0, 0]], np.zeros((0, 3)), 0.1).shape == (0, 3)
    with pytest.raises(ValueError):
        oracle.sl([[0, 0, 0]], [1.0], [[1, 0, 0]], [[1, 0, 0]], 0.0)
    with pytest.raises(ValueError):
        oracle.sl([[0, 0, 0]], [1.0], [[1, 0, 0]], [[1, 0, 0]], 0.1, mu=0.0)
    with pytest.raises(ValueError):
        oracle.sl([[0, 0, 0]], [1.0], [[1, 0, 0]], [[1, 0, 0], [2, 0, 0], [3, 0, 0]], [0.1, 0.2])


def test_sl_coincident_nodes_even_m():
    """Even m: nodes of different patches coincide (r = 0 or ~1e-16); the
    series and the r = 0 limit handle them."""
    s = ci.make_surface(ci.Sphere(1.0), 16)
    d = np.linalg.norm(s.X[:, None, :] - s.X[None, :, :], axis=-1)
    np.fill_diagonal(d, 1.0)
    assert d.min() < 1e-15
    f = np.zeros((s.N, 3))
    f[:, 2] = 1.0
    u = oracle.sl(s.X, s.w, f, s.X, 2 * s.h)
    assert np.all(np.isfinite(u))
    assert np.abs(u - np.array([0, 0, 2.0 / 3.0])).max() < 1e-3


def test_sl_threads_do_not_change_results():
    w = ci.rbc_workload(m=9)
    s = w.surface
    u1 = oracle.sl(s.X, s.w, w.f, w.targets, w.delta, threads=1)
    u4 = oracle.sl(s.X, s.w, w.f, w.targets, w.delta, threads=4)
    assert np.array_equal(u1, u4)
