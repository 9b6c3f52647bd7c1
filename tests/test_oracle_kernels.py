"""Pins for the oracle's smoothing factors s1, s2, s3 and their series.

Sec. 3.4 prints s1, s2 and the r -> 0 limits of s1/r and s2/r^3; the
double-layer factor s3 is the reading recorded in the design notes (the
paper prints no double-layer formula).
"""

import math

import numpy as np
import pytest

import oracle
from conftest import read_golden

SQPI = math.sqrt(math.pi)


@pytest.mark.parametrize("row", read_golden("kernel_limits.txt"))
def test_small_r_limits_match_paper(row):
    name, num, den, power = row[0], float(row[1]), float(row[2]), int(row[3])
    which = {"s1_over_r": 1, "s2_over_r3": 2}[name]
    limit = num / (den * SQPI)
    # k_i(0) * delta^{-power} is the limit of s_i(r/delta) / r^power
    assert oracle.kernel_factor(which, [0.0])[0] == pytest.approx(limit, rel=1e-15)
    for delta in (0.01, 0.3, 2.0):
        k = oracle.kernel_factor(which, [1e-9 / delta])[0] / delta ** power
        assert k == pytest.approx(limit / delta ** power, rel=1e-12)


def test_double_layer_factor_is_fifth_order_at_zero():
    # s3(p) = (128 / (15 sqrt(pi))) p^5 + O(p^7): the p, p^3 terms cancel.
    assert oracle.kernel_factor(3, [0.0])[0] == pytest.approx(128.0 / (15.0 * SQPI), rel=1e-15)


def test_series_agree_with_high_precision_closed_forms():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60

    def s(which, p):
        p = mp.mpf(p)
        e = mp.exp(-p * p) / mp.sqrt(mp.pi)
        if which == 1:
            return (mp.erf(p) - mp.mpf(2) / 3 * p * (2 * p ** 2 - 5) * e) / p
        if which == 2:
            return (mp.erf(p) - mp.mpf(2) / 3 * p * (4 * p ** 4 - 14 * p ** 2 + 3) * e) / p ** 3
        return (mp.erf(p) - mp.mpf(2) / 9 * p * (8 * p ** 6 - 36 * p ** 4 + 6 * p ** 2 + 9) * e) / p ** 5

    rhos = np.concatenate([np.geomspace(1e-4, 0.99, 25), np.linspace(1.0, 8.0, 30)])
    for which in (1, 2, 3):
        got = oracle.kernel_factor(which, rhos)
        ref = np.array([float(s(which, p)) for p in rhos])
        assert np.max(np.abs(got / ref - 1)) < 5e-15, which
        # the series alone is accurate on [0, 1.2]
        small = rhos[rhos < 1.2]
        ser = oracle.kernel_factor(which, small, branch="series")
        refs = np.array([float(s(which, p)) for p in small])
        assert np.max(np.abs(ser / refs - 1)) < 5e-15, which


def test_closed_form_loses_digits_at_small_rho_but_series_does_not():
    # why the oracle switches to the series below p = 1
    p = np.array([1e-3])
    closed = oracle.kernel_factor(2, p, branch="closed")[0]
    series = oracle.kernel_factor(2, p, branch="series")[0]
    assert abs(closed / series - 1) > 1e-12
    assert series == pytest.approx(32 / (3 * SQPI), rel=1e-5)


def test_far_field_factors_tend_to_one():
    p = np.array([7.0, 8.0, 12.0, 30.0])  # e^{-49} p^7 ~ 1e-15 at p = 7
    for which, power in ((1, 1), (2, 3), (3, 5)):
        k = oracle.kernel_factor(which, p)
        # s_i -> 1, so k_i(p) -> p^{-power}
        assert np.allclose(k * p ** power, 1.0, rtol=0, atol=1e-14)
    assert oracle.smoothing(1, [10.0])[0] == 1.0


def test_continuity_across_series_switch():
    for which in (1, 2, 3):
        lo = oracle.kernel_factor(which, [np.nextafter(1.0, 0.0)])[0]
        hi = oracle.kernel_factor(which, [1.0])[0]
        assert abs(lo / hi - 1) < 1e-14


def test_far_cutoff_tails_at_the_default_rho_c():
    """The plain Stokeslet/stresslet used at r/delta >= rho_c omits 1 - s_i,
    largest at rho_c. The library documents these fractions for rho_c = 5
    (its default) and 5.5: 1.2e-9 (s1), 5.6e-8 (s2), 8.9e-7 (s3) at 5;
    4.9e-10 (s2), 9.5e-9 (s3) at 5.5; each falls monotonically beyond."""
    tail = {i: 1.0 - oracle.smoothing(i, [5.0, 5.5, 6.0]) for i in (1, 2, 3)}
    assert tail[1][0] == pytest.approx(1.18e-9, rel=0.01)
    assert tail[2][0] == pytest.approx(5.62e-8, rel=0.01)
    assert tail[3][0] == pytest.approx(8.94e-7, rel=0.01)
    assert tail[2][1] == pytest.approx(4.88e-10, rel=0.01)
    assert tail[3][1] == pytest.approx(9.48e-9, rel=0.01)
    for i in (1, 2, 3):
        assert tail[i][0] > tail[i][1] > tail[i][2] > 0
    # the leading behaviour: 1 - s_i ~ c p^(2i+1) e^{-p^2} / sqrt(pi) with
    # c = 4/3, 8/3, 16/9 (the top term of each polynomial times p); erfc p is
    # smaller by a factor ~ p^(2i+2)
    p = 5.0
    for i, c in ((1, 4 / 3), (2, 8 / 3), (3, 16 / 9)):
        lead = c * p ** (2 * i + 1) * math.exp(-p * p) / SQPI
        assert tail[i][0] == pytest.approx(lead, rel=0.2)
