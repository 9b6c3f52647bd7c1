"""The FP32 smoothing factors of the pair kernels (Sec. 3.4, and reading R7 for
the stresslet's s3) are written as 1 - exp(-rho^2) (E(rho) + polynomial), with
erf(rho) = 1 - exp(-rho^2) E(rho) and E(rho) = exp(rho^2) erfc(rho) fitted in
csrc/sk_erfc_scaled.h by csrc/fit_erfc_scaled.py.

Checks, without a GPU: the header holds that script's fit; the fit is within
2e-8 of E in double precision; and the kernels' FP32 formulas, evaluated here
in float32 with the header's coefficients, stay within FP32 rounding of the
exact factors over the smoothing range [0.25, 8] (the exact ones from
scipy.special.erf in double precision).
"""

import importlib.util
import os
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2310_13908_gb300", "csrc")


def load_script():
    spec = importlib.util.spec_from_file_location("fit_erfc_scaled",
                                                  os.path.join(CSRC, "fit_erfc_scaled.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def header_coefficients():
    """c_0 .. c_8 as written in the header (the Horner nest lists c_8 first)."""
    text = open(os.path.join(CSRC, "sk_erfc_scaled.h")).read()
    body = text[text.index("return t *"):]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals[::-1])


def test_header_holds_the_fit():
    fit = load_script()
    c, err = fit.fit()
    h = header_coefficients()
    assert h.shape == c.shape
    np.testing.assert_allclose(h, c, rtol=1e-8, atol=1e-10)
    assert err <= 2e-8


def smoothing_f32(rho):
    """The kernels' FP32 smoothing factors (s1, s2, s3) at float32 rho."""
    f = np.float32
    c = header_coefficients().astype(f)
    t = (f(1) / (f(1) + f(0.4) * rho)).astype(f)
    P = np.full_like(t, c[-1])
    for k in range(len(c) - 2, -1, -1):
        P = (P * t + c[k]).astype(f)
    E = (t * P).astype(f)
    p2 = (rho * rho).astype(f)
    e = np.exp(-p2.astype(np.float64)).astype(f)
    cr = (f(2.0 / 3.0 / np.sqrt(np.pi)) * rho).astype(f)
    s1 = (f(1) - e * (cr * (f(2) * p2 - f(5)) + E)).astype(f)
    s2 = (f(1) - e * (cr * ((f(4) * p2 - f(14)) * p2 + f(3)) + E)).astype(f)
    c3 = (f(2.0 / 9.0 / np.sqrt(np.pi)) * rho).astype(f)
    s3 = (f(1) - e * (c3 * (((f(8) * p2 - f(36)) * p2 + f(6)) * p2 + f(9)) + E)).astype(f)
    return s1, s2, s3


def smoothing_exact(rho):
    r = rho.astype(np.float64)
    p = r * r
    g = np.exp(-p) / np.sqrt(np.pi)
    er = special.erf(r)
    s1 = er - (2.0 / 3.0) * r * (2 * p - 5) * g
    s2 = er - (2.0 / 3.0) * r * ((4 * p - 14) * p + 3) * g
    s3 = er - (2.0 / 9.0) * r * (((8 * p - 36) * p + 6) * p + 9) * g
    return s1, s2, s3


def test_fp32_factors_within_rounding():
    rho = np.linspace(0.25, 8.0, 200001).astype(np.float32)
    got = smoothing_f32(rho)
    ref = smoothing_exact(rho)
    # largest values: s1 ~ 1.2, s2 ~ 1.6, s3 ~ 2.4; a few float32 ulps of them
    for g, r, bound in zip(got, ref, (5e-7, 5e-7, 8e-7)):
        assert np.abs(g - r).max() <= bound
    # the factors reach 1 beyond the smoothing range
    assert np.all(np.abs(np.array([x[-1] for x in got]) - 1.0) < 1e-6)


def test_a_wrong_coefficient_is_caught():
    """A planted mistake in one coefficient (as a typo in the header would
    make) moves the factors by far more than rounding."""
    f = np.float32
    c = header_coefficients()
    c[3] *= 1.001
    rho = np.linspace(0.25, 8.0, 20001).astype(f)
    t = (1.0 / (1.0 + 0.4 * rho.astype(np.float64)))
    E = t * np.polynomial.polynomial.polyval(t, c)
    err = np.abs(E - special.erfcx(rho.astype(np.float64))).max()
    assert err > 1e-5
