"""Oracle double layer: pinned to the constant-density identities and rates."""

import math

import numpy as np
import pytest

import capsule_inputs as ci
import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.DL_PINS, ids=lambda p: p.__name__)
def test_dl_pin(pin):
    pin(oracle.default())


def test_dl_brute_force_tiny_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(31)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 4)
    q = rng.standard_normal((s.N, 3))
    delta = 1.5 * s.h
    u = oracle.dl(s.X, s.w, s.n, q, s.X, delta)
    sq = mp.sqrt(mp.pi)
    for t in range(s.N):
        acc = [mp.mpf(0)] * 3
        for j in range(s.N):
            if s.w[j] == 0:
                continue
            d = [mp.mpf(s.X[t, c]) - mp.mpf(s.X[j, c]) for c in range(3)]
            r = mp.sqrt(sum(x * x for x in d))
            if r == 0:
                continue
            p = r / delta
            s3 = mp.erf(p) - mp.mpf(2) / 9 * p * (8 * p ** 6 - 36 * p ** 4 + 6 * p * p + 9) \
                * mp.exp(-p * p) / sq
            dq = sum(d[c] * mp.mpf(q[j, c]) for c in range(3))
            dn = sum(d[c] * mp.mpf(s.n[j, c]) for c in range(3))
            for c in range(3):
                acc[c] += mp.mpf(s.w[j]) * (-6) * dq * dn * d[c] * s3 / r ** 5
        ref = np.array([float(x / (8 * mp.pi)) for x in acc])
        assert np.allclose(u[t], ref, rtol=1e-12, atol=1e-14 * max(1.0, np.abs(ref).max()))


def test_dl_linearity_and_rotation():
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 7)
    rng = np.random.default_rng(6)
    q1, q2 = rng.standard_normal((2, s.N, 3))
    u1 = oracle.dl(s.X, s.w, s.n, q1, s.X, 0.4)
    u2 = oracle.dl(s.X, s.w, s.n, q2, s.X, 0.4)
    assert np.allclose(oracle.dl(s.X, s.w, s.n, q1 - 3 * q2, s.X, 0.4), u1 - 3 * u2,
                       rtol=1e-12, atol=1e-13)
    Q = ci.random_rotation(rng)
    ur = oracle.dl(s.X @ Q.T, s.w, s.n @ Q.T, q1 @ Q.T, s.X @ Q.T, 0.4)
    assert np.allclose(ur, u1 @ Q.T, rtol=1e-10, atol=1e-12)


def test_dl_validation():
    with pytest.raises(ValueError):
        oracle.dl([[0, 0, 0]], [1.0], [[0, 0, 1]], [[1, 0, 0]], [[1, 0, 0]], -1.0)
