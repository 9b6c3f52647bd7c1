"""Smooth random densities on the capsule (evaluated on the sphere preimage).

A density of spherical-harmonic degree <= lmax is sum_{l, m} a_lm Y_lm(x0)
per component, with real orthonormal Y_lm and a_lm ~ N(0, 1) / (l + 1).
Because it is evaluated at the preimage x0 = phi^{-1}(x), the field is smooth
on any surface phi(S^2).
"""

from __future__ import annotations

import math

import numpy as np


def real_sph_harm(lmax: int, x0: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics up to degree lmax at unit vectors x0.

    Returns shape (N, (lmax+1)^2); column l*l + l + m holds Y_lm, m = -l..l
    (cos(m phi) for m > 0, sin(|m| phi) for m < 0). Associated Legendre
    functions come from the standard three-term recurrence in l.
    """
    x0 = np.asarray(x0, dtype=np.float64)
    z = np.clip(x0[:, 2], -1.0, 1.0)
    ph = np.arctan2(x0[:, 1], x0[:, 0])
    sint = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    N = x0.shape[0]
    out = np.empty(((lmax + 1) ** 2, N))  # rows are contiguous; returned transposed
    for mm in range(lmax + 1):
        # P_mm = (-1)^m (2m-1)!! sin^m
        pmm = ((-1.0) ** mm * _double_factorial(2 * mm - 1)) * sint ** mm
        P = {mm: pmm}
        if mm + 1 <= lmax:
            P[mm + 1] = z * (2 * mm + 1) * pmm
        for ll in range(mm + 2, lmax + 1):
            P[ll] = ((2 * ll - 1) * z * P[ll - 1] - (ll + mm - 1) * P[ll - 2]) / (ll - mm)
        if mm > 0:
            cm, sm = np.cos(mm * ph), np.sin(mm * ph)
        for ll in range(mm, lmax + 1):
            norm = math.sqrt((2 * ll + 1) / (4 * math.pi)
                             * math.factorial(ll - mm) / math.factorial(ll + mm))
            if mm == 0:
                np.multiply(P[ll], norm, out=out[ll * ll + ll])
            else:
                a = (math.sqrt(2.0) * norm) * P[ll]
                np.multiply(a, cm, out=out[ll * ll + ll + mm])
                np.multiply(a, sm, out=out[ll * ll + ll - mm])
    return out.T


def _double_factorial(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def sh_density(x0: np.ndarray, rng: np.random.Generator, lmax: int = 8,
               components: int = 3) -> np.ndarray:
    """Random smooth field of degree <= lmax, shape (N, components)."""
    Y = real_sph_harm(lmax, x0)
    deg = np.concatenate([[l] * (2 * l + 1) for l in range(lmax + 1)])
    coef = rng.standard_normal(((lmax + 1) ** 2, components)) / (deg[:, None] + 1.0)
    return Y @ coef


def gaussian_noise(n: int, sigma: float, rng: np.random.Generator,
                   components: int = 3) -> np.ndarray:
    """i.i.d. N(0, sigma^2) per node and component."""
    return sigma * rng.standard_normal((n, components))
