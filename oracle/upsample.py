"""Four-times upsampled single layer (Sec. 3.4, "Upsampling"), written out
plainly in FP64. Test infrastructure (see oracle/__init__.py).

The single layer of Eq. regstokes is evaluated with sources on the upsampled
grid of order q m (q = 4; (q m - 1)^2 nodes per patch, N_up = 6 (q m - 1)^2):
  X_u = I_u X, F_u = I_u F, W_u = I_u W (cubic-spline interpolation on each
  patch), psi_u = the POU at the fine nodes, weights psi_u W_u h_u^2
  (h_u = pi / (q m), Eq. smoothint), delta_u from Eq. regparam on the fine
  grid (C = 1, per patch);
and then brought back to the m-th order grid by I_d.

Readings:
  * I_u is the patch's tensor-product not-a-knot cubic spline (the same
    interpolant as the patch extension of Sec. 3.5) evaluated at the fine
    nodes, continued by its end pieces for fine nodes beyond the first/last
    coarse node (their psi_u is 0 there, so they carry no weight).
  * Every coarse node is also a fine node (j pi / m = q j pi / (q m)), and a
    spline interpolant reproduces the values at its own nodes, so I_d returns
    the fine-grid potential at the coarse nodes. The oracle therefore
    evaluates the sum only at the coarse nodes (targets) with the fine
    sources; the target's delta is delta_u of its patch.
"""

from __future__ import annotations

import numpy as np

import capsule_inputs as ci
from capsule_inputs.geometry import chart, pou_all

from . import membrane as mb
from . import sl as oracle_sl

FACTOR = 4


def fine_grid(m: int, q: int = FACTOR):
    """(patch, u, v) of the fine nodes, patch-major, then u index, then v."""
    mu = q * m
    h = np.pi / mu
    jj, kk = np.meshgrid(np.arange(1, mu), np.arange(1, mu), indexing="ij")
    u, v = (jj * h).ravel(), (kk * h).ravel()
    return mu, u, v


def upsample(m: int, G: np.ndarray, q: int = FACTOR) -> np.ndarray:
    """I_u: node values G (6 (m-1)^2, F) -> fine-grid values (6 (q m - 1)^2, F)."""
    G = np.asarray(G, dtype=np.float64)
    flat = G.reshape(G.shape[0], -1)
    Gp = flat.reshape(6, m - 1, m - 1, -1)
    _, u, v = fine_grid(m, q)
    out = np.concatenate([mb.interpolate(m, Gp[p], u, v) for p in range(6)], axis=0)
    return out.reshape((out.shape[0],) + G.shape[1:])


def fine_pou(m: int, q: int = FACTOR) -> np.ndarray:
    """psi_u: the POU of each fine node's own patch (Eq. pou0)."""
    _, u, v = fine_grid(m, q)
    return np.concatenate([pou_all(chart(p, u, v))[:, p - 1] for p in range(1, 7)])


def fine_delta_star(m: int, Xu: np.ndarray, q: int = FACTOR, C: float = 1.0) -> np.ndarray:
    """delta_u per fine node: Eq. regparam on the fine grid."""
    surf = ci.make_surface(ci.Sphere(1.0), q * m)
    surf.X = Xu
    return ci.delta_star(surf, C)


def sl_upsampled(m: int, X: np.ndarray, W: np.ndarray, f: np.ndarray, mu: float = 1.0,
                 q: int = FACTOR, targets=None) -> np.ndarray:
    """S[f] at the m-th order nodes X by the upsampled sum; W is the area
    element at the nodes (e.g. from the derivative scheme). targets: optional
    indices of the nodes to evaluate (default all)."""
    Xu = upsample(m, X, q)
    Wu = upsample(m, W, q)
    Fu = upsample(m, f, q)
    hu = np.pi / (q * m)
    wu = fine_pou(m, q) * Wu * hu * hu
    du_fine = fine_delta_star(m, Xu, q)
    # delta of a coarse target = delta_u of its patch (constant per patch)
    n = m - 1
    d_patch = du_fine.reshape(6, -1)[:, 0]
    d_tgt = np.repeat(d_patch, n * n)
    idx = np.arange(X.shape[0]) if targets is None else np.asarray(targets)
    return oracle_sl(Xu, wu, Fu, X[idx], d_tgt[idx], mu)
