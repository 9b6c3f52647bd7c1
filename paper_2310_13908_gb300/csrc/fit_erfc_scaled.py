"""Coefficients of the FP32 scaled complementary error function of the pair
kernels' smoothing factors, written to sk_erfc_scaled.h.

The smoothing factors of Sec. 3.4 (and of the stresslet) are erf(rho) minus a
polynomial times exp(-rho^2). With erf = 1 - exp(-rho^2) E(rho), where
E(rho) = exp(rho^2) erfc(rho), each factor becomes 1 - exp(-rho^2) (E(rho) +
polynomial): one exponential and one smooth, bounded function, instead of an
error function and an exponential. E is fitted here, by least squares on
Chebyshev points of [0.2, 8.5] (every rho the kernels smooth at lies in
[rho_T, rho_c] with 0 < rho_T and rho_c <= 8), in the variable
t = 1 / (1 + 0.4 rho): E(rho) ~ t * sum_k c_k t^k, degree 8. The reference
values come from scipy.special.erfcx (double precision).

Run from this directory: python fit_erfc_scaled.py (rewrites the header).
"""

import os

import numpy as np

A = 0.4
DEGREE = 8
LO, HI = 0.2, 8.5
N_FIT = 4000


def fit():
    """Coefficients c_0 .. c_DEGREE (float64) and the largest absolute error
    of the float64 fit on a fine grid of [LO, HI]."""
    from scipy.special import erfcx
    k = np.arange(N_FIT)
    r = np.cos(np.pi * (k + 0.5) / N_FIT) * (HI - LO) / 2 + (HI + LO) / 2
    t = 1.0 / (1.0 + A * r)
    c = np.polynomial.polynomial.polyfit(t, erfcx(r) / t, DEGREE)
    rr = np.linspace(LO, HI, 200001)
    tt = 1.0 / (1.0 + A * rr)
    err = np.abs(tt * np.polynomial.polynomial.polyval(tt, c) - erfcx(rr)).max()
    return c, float(err)


def header_text(c, err):
    horner = "%.9ef" % c[DEGREE]
    for k in range(DEGREE - 1, -1, -1):
        horner = "fmaf(%s, t, %.9ef)" % (horner, c[k])
    lines = [
        "// Generated by fit_erfc_scaled.py (least-squares fit; do not edit by hand).",
        "// E(rho) = exp(rho^2) erfc(rho) for 0.2 <= rho <= 8.5, as t * P(t) with",
        "// t = 1 / (1 + %.1f rho), P of degree %d; largest absolute error of the fit" % (A, DEGREE),
        "// in double precision: %.1e. The pair kernels' smoothing factors use it." % err,
        "#pragma once",
        "",
        "__device__ __forceinline__ float erfc_scaled(float rho) {",
        "  float t;",
        '  asm("rcp.approx.ftz.f32 %%0, %%1;" : "=f"(t) : "f"(fmaf(%.1ff, rho, 1.f)));' % A,
        "  return t * %s;" % horner,
        "}",
        "",
    ]
    # wrap the long Horner line at its fmaf boundaries
    out = []
    for line in lines:
        if len(line) <= 100:
            out.append(line)
            continue
        parts = line.split(", t, ")
        cur = parts[0]
        for p in parts[1:]:
            if len(cur) > 80:
                out.append(cur + ",")
                cur = "             t, " + p
            else:
                cur += ", t, " + p
        out.append(cur)
    return "\n".join(out)


if __name__ == "__main__":
    c, err = fit()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sk_erfc_scaled.h")
    with open(path, "w") as fh:
        fh.write(header_text(c, err))
    print("wrote", path, "fit error %.2e" % err)
