"""Single-level kernel-independent FMM for the single layer (Sec. 5), written
out plainly in FP64 NumPy. Test infrastructure (see oracle/__init__.py).

Steps, in the paper's order:
  1. k-means clustering of the source points (k clusters);
  2. per cluster, an enclosing cube carrying equivalent sources on a regular
     grid of its surface, and a larger check cube; the equivalent densities
     reproduce, on the check surface, the potential of the cluster's points;
  3. box against box: the points of a box take the direct (regularized) sum
     over the points of the neighbouring boxes and the equivalent sources of
     the non-neighbouring ones.

Readings (the paper gives no more detail):
  * Sources with zero weight are dropped first (they contribute exactly 0).
  * k-means: Lloyd iterations from caller-given initial centres; a point
    goes to its nearest centre, by the squared distance (dx^2 + dy^2) + dz^2
    (lowest index on ties); a centre moves to the mean of its points (an
    empty cluster keeps its centre); the clusters are those of the final
    assignment to the final centres.
  * Source boxes: the cube of a cluster has its centre at the midpoint of
    the points' bounding box and half width a = half the largest extent.
    Equivalent cube: half width 1.05 a; check cube: 2.95 a (the radii of the
    kernel-independent FMM the paper builds on). Surface grids: p points per
    edge (6p^2 - 12p + 8).
  * Equivalent densities: Tikhonov-regularized least squares,
    min |K phi - u_check|^2 + alpha^2 |phi|^2 with alpha = 1e-8 |K|_F, K the
    plain-Stokeslet matrix from equivalent to check points. (A truncated
    pseudo-inverse does no better here; this one scales exactly with the
    cube size, phi(a) = a phi(1).)
  * Target boxes: the targets need not be nodes (off-surface probes), so
    each target joins the box of its nearest final centre, by the same rule
    as the points; a target box is the bounding box of its targets, with the
    largest delta among them.
  * Neighbouring boxes: source cluster j is a neighbour of target box i
    unless the whole target box lies outside j's check cube (where the
    equivalent sources reproduce the cluster's potential) and at least
    7 delta_i from j's cube (where the regularized kernel of every source of
    the cluster equals the plain one to double precision).
"""

from __future__ import annotations

import numpy as np

from . import plain_stokeslet
from . import sl as oracle_sl

R_EQUIV = 1.05
R_CHECK = 2.95
RHO_FAR = 7.0
TIKHONOV = 1e-8


def nearest_centre(points: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Index of the nearest centre of every point (lowest index on ties)."""
    d = points[:, None, :] - c[None, :, :]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    return np.argmin(d2, axis=1)   # first minimum: lowest index on ties


def kmeans(points: np.ndarray, centers0: np.ndarray, iters: int):
    """Lloyd iterations; returns (centers, labels of the final assignment)."""
    c = np.array(centers0, dtype=np.float64, copy=True)
    for _ in range(iters):
        lab = nearest_centre(points, c)
        for j in range(len(c)):
            sel = lab == j
            if np.any(sel):
                c[j] = points[sel].mean(axis=0)
    return c, nearest_centre(points, c)


def cube_surface(p: int) -> np.ndarray:
    """Regular grid points of the surface of [-1, 1]^3, p per edge."""
    t = np.linspace(-1.0, 1.0, p)
    pts = [(x, y, z) for x in t for y in t for z in t
           if abs(x) == 1.0 or abs(y) == 1.0 or abs(z) == 1.0]
    return np.array(pts)


def stokeslet_matrix(targets: np.ndarray, sources: np.ndarray) -> np.ndarray:
    """Plain Stokeslet I/r + d d^T / r^3 (without 1/(8 pi mu)), (3 nt, 3 ns)."""
    d = targets[:, None, :] - sources[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    G = np.eye(3)[None, None] / r[..., None, None] + d[..., :, None] * d[..., None, :] / (
        r ** 3)[..., None, None]
    return G.transpose(0, 2, 1, 3).reshape(3 * len(targets), 3 * len(sources))


def boxes(points: np.ndarray, labels: np.ndarray, k: int):
    """Centre and half width of each cluster's cube."""
    cen = np.zeros((k, 3))
    a = np.zeros(k)
    for j in range(k):
        sel = labels == j
        if np.any(sel):
            lo, hi = points[sel].min(axis=0), points[sel].max(axis=0)
            cen[j] = 0.5 * (lo + hi)
            a[j] = max(0.5 * float(np.max(hi - lo)), 1e-12)
    return cen, a


def equivalent_densities(points, weights, f, labels, cen, a, p):
    """Per cluster: equivalent points and densities (plain kernel, no 1/(8 pi mu))."""
    unit = cube_surface(p)
    eq_pts, eq_den = [], []
    for j in range(len(cen)):
        sel = labels == j
        E = cen[j] + R_EQUIV * a[j] * unit
        if not np.any(sel):
            eq_pts.append(E)
            eq_den.append(np.zeros((len(unit), 3)))
            continue
        C = cen[j] + R_CHECK * a[j] * unit
        g = weights[sel, None] * f[sel]
        u_check = stokeslet_matrix(C, points[sel]) @ g.ravel()
        K = stokeslet_matrix(C, E)
        alpha = TIKHONOV * np.linalg.norm(K)
        A = np.vstack([K, alpha * np.eye(K.shape[1])])
        phi = np.linalg.lstsq(A, np.concatenate([u_check, np.zeros(K.shape[1])]), rcond=None)[0]
        eq_pts.append(E)
        eq_den.append(phi.reshape(-1, 3))
    return eq_pts, eq_den


def neighbours(lo, hi, delta_i, cen, a):
    """Neighbour flags of one target box [lo, hi] (largest delta delta_i)
    against every source cluster cube (cen, a): True where the direct sum
    is required."""
    outside_check = np.any((lo[None] > cen + R_CHECK * a[:, None]) |
                           (hi[None] < cen - R_CHECK * a[:, None]), axis=1)
    g = np.maximum(np.maximum(lo[None] - (cen + a[:, None]), (cen - a[:, None]) - hi[None]), 0.0)
    gap2 = (g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1]) + g[:, 2] * g[:, 2]
    far = outside_check & (gap2 >= (RHO_FAR * delta_i) * (RHO_FAR * delta_i))
    return ~far


def far_field(T, E, phi):
    """Plain Stokeslet sum (without 1/(8 pi mu)) of equivalent sources E with
    densities phi at the points T: sum_e phi_e / r + (phi_e . d) d / r^3."""
    return plain_stokeslet(E, phi, T)


def plan(src, w, tgt, delta, centers0, iters):
    """The FMM's discrete decisions: active sources, k-means centres and
    labels, cluster cubes, target boxes and the neighbour matrix
    near[i, j] (target box i, source cluster j)."""
    src = np.asarray(src, np.float64)
    tgt = np.asarray(tgt, np.float64)
    w = np.asarray(w, np.float64)
    delta = np.broadcast_to(np.asarray(delta, np.float64), (len(tgt),))
    act = w != 0.0           # zero weights contribute exactly nothing
    k = len(centers0)
    centers, labels = kmeans(src[act], centers0, iters)
    cen, a = boxes(src[act], labels, k)
    tlab = nearest_centre(tgt, centers)
    near = np.zeros((k, k), dtype=bool)
    for i in range(k):
        ti = np.flatnonzero(tlab == i)
        if len(ti):
            T = tgt[ti]
            near[i] = neighbours(T.min(axis=0), T.max(axis=0), float(delta[ti].max()), cen, a)
    return {"act": act, "centers": centers, "labels": labels, "cen": cen, "a": a,
            "tlab": tlab, "near": near, "delta": delta}


def sl_fmm(src, w, f, tgt, delta, mu, centers0, iters, p):
    """S[f] at the targets by the single-level FMM."""
    pl = plan(src, w, tgt, delta, centers0, iters)
    act, labels, cen, a, tlab, near = (pl[x] for x in ("act", "labels", "cen", "a", "tlab",
                                                       "near"))
    delta = pl["delta"]
    src = np.asarray(src, np.float64)[act]
    w = np.asarray(w, np.float64)[act]
    f = np.asarray(f, np.float64)[act]
    tgt = np.asarray(tgt, np.float64)
    k = len(cen)
    eq_pts, eq_den = equivalent_densities(src, w, f, labels, cen, a, p)
    u = np.zeros((len(tgt), 3))
    scale = 1.0 / (8.0 * np.pi * mu)
    for i in range(k):
        ti = np.flatnonzero(tlab == i)
        if len(ti) == 0:
            continue
        T = tgt[ti]
        far_j = [j for j in range(k) if not near[i, j] and np.any(labels == j)]
        sel = near[i][labels]           # the points of the neighbouring clusters
        if np.any(sel):
            u[ti] += oracle_sl(src[sel], w[sel], f[sel], T, delta[ti], mu)
        if far_j:
            E = np.concatenate([eq_pts[j] for j in far_j])
            phi = np.concatenate([eq_den[j] for j in far_j])
            u[ti] += scale * far_field(T, E, phi)
    return u
