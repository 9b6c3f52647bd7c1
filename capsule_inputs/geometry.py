"""Six-patch atlas, partition of unity, grids and closed-form surface maps.

Paper references (section / equation names of arXiv 2310.13908):
  * charts eta_i^0 on U_i = (0, pi)^2 ............ Sec. 3.1, Eq. param_maps
  * bump b(r) and POU psi_i^0, r0 = 5 pi / 12 .... Sec. 3.1, Eq. pou0
  * psi_i = psi_i^0 o phi^{-1} ................... Sec. 3.1, Eq. pou
  * m-th order grid U_{jk} = (j pi/m, k pi/m) .... Sec. 3.2, Eqs. sph_grid, grid
  * ellipsoid map phi = beta o beta0^{-1} ........ Sec. 3.2, Eq. sphangles_ellip
  * area element W = |x_u x x_v|, n = x_u x x_v / W  Appendix, Table diff_formulas
  * quadrature weight psi * W * h_m^2 ............ Sec. 3.3, Eq. smoothint
  * delta* (max neighbour distance per patch) .... Sec. 3.4, Eq. regparam

The paper computes tangents by finite differences; here they are closed-form
(chain rule through phi), which is what an input generator needs.
"""

from __future__ import annotations

import functools
from dataclasses import dataclass, field

import numpy as np

# r0 = 5 pi / 12 (Sec. 3.1, below Eq. pou0; Appendix "choice of r0").
R0_POU = 5.0 * np.pi / 12.0

N_PATCHES = 6


def chart(i: int, u, v) -> np.ndarray:
    """eta_i^0(u, v) on the unit sphere, i = 1..6 (Sec. 3.1, Eq. param_maps)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    su, cu, sv, cv = np.sin(u), np.cos(u), np.sin(v), np.cos(v)
    if i == 1:
        c = (su * cv, su * sv, cu)
    elif i == 2:
        c = (-su * cv, -su * sv, cu)
    elif i == 3:
        c = (su * sv, -su * cv, cu)
    elif i == 4:
        c = (-su * sv, su * cv, cu)
    elif i == 5:
        c = (su * cv, -cu, su * sv)
    elif i == 6:
        c = (su * cv, cu, -su * sv)
    else:
        raise ValueError(f"chart index must be 1..6, got {i}")
    return np.stack(np.broadcast_arrays(*c), axis=-1)


def chart_tangents(i: int, u, v):
    """(d eta_i^0 / du, d eta_i^0 / dv), differentiated from Eq. param_maps."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    su, cu, sv, cv = np.sin(u), np.cos(u), np.sin(v), np.cos(v)
    z = np.zeros_like(su * cv)
    if i == 1:
        du, dv = (cu * cv, cu * sv, -su), (-su * sv, su * cv, z)
    elif i == 2:
        du, dv = (-cu * cv, -cu * sv, -su), (su * sv, -su * cv, z)
    elif i == 3:
        du, dv = (cu * sv, -cu * cv, -su), (su * cv, su * sv, z)
    elif i == 4:
        du, dv = (-cu * sv, cu * cv, -su), (-su * cv, -su * sv, z)
    elif i == 5:
        du, dv = (cu * cv, su, cu * sv), (-su * sv, z, su * cv)
    elif i == 6:
        du, dv = (cu * cv, -su, -cu * sv), (-su * sv, z, -su * cv)
    else:
        raise ValueError(f"chart index must be 1..6, got {i}")
    return (np.stack(np.broadcast_arrays(*du), axis=-1),
            np.stack(np.broadcast_arrays(*dv), axis=-1))


# Patch centres eta_i^0(pi/2, pi/2) (Sec. 3.1, Eq. pou0).
CHART_CENTERS = np.stack([chart(i, np.pi / 2, np.pi / 2) for i in range(1, 7)])


def bump(r) -> np.ndarray:
    """b(r) = exp(2 exp(-1/|r|) / (|r| - 1)) for |r| < 1, else 0 (Sec. 3.1)."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    inside = r < 1.0
    ri = r[inside]
    with np.errstate(divide="ignore", over="ignore", under="ignore"):
        e = np.where(ri > 0.0, np.exp(-1.0 / np.where(ri > 0.0, ri, 1.0)), 0.0)
        out[inside] = np.exp(2.0 * e / (ri - 1.0))
    return out


def great_circle(x0: np.ndarray, y0: np.ndarray) -> np.ndarray:
    """Great-circle distance between unit vectors (arccos of the clamped dot)."""
    dot = np.clip(np.sum(x0 * y0, axis=-1), -1.0, 1.0)
    return np.arccos(dot)


def pou_all(x0: np.ndarray, r0: float = R0_POU) -> np.ndarray:
    """psi_i^0(x0) for all six patches, shape (..., 6) (Sec. 3.1, Eq. pou0)."""
    b = np.stack([bump(great_circle(x0, CHART_CENTERS[i]) / r0) for i in range(N_PATCHES)],
                 axis=-1)
    return b / np.sum(b, axis=-1, keepdims=True)


def pou_weight(i: int, x0: np.ndarray, r0: float = R0_POU) -> np.ndarray:
    """psi_i^0(x0) for one patch i = 1..6."""
    return pou_all(x0, r0)[..., i - 1]


def patch_grid(m: int):
    """m-th order grid of all six patches (Sec. 3.2, Eq. sph_grid).

    Returns (patch, j, k, u, v, x0) with N = 6 (m-1)^2 entries, ordered
    patch-major, then j (u index), then k (v index); patch in 1..6 and
    j, k in 1..m-1, u = j pi/m, v = k pi/m, x0 = eta_patch^0(u, v).
    """
    if m < 2:
        raise ValueError("m must be >= 2")
    n = m - 1
    jj, kk = np.meshgrid(np.arange(1, m), np.arange(1, m), indexing="ij")
    jj = jj.ravel()
    kk = kk.ravel()
    h = np.pi / m
    patch = np.repeat(np.arange(1, 7), n * n)
    j = np.tile(jj, 6)
    k = np.tile(kk, 6)
    u = j * h
    v = k * h
    x0 = np.empty((6 * n * n, 3))
    for i in range(1, 7):
        sl = slice((i - 1) * n * n, i * n * n)
        x0[sl] = chart(i, u[sl], v[sl])
    return patch, j, k, u, v, x0


# --------------------------------------------------------------------------
# Surface maps phi : S^2 -> gamma, with their Jacobians (3x3, acting on R^3).
# --------------------------------------------------------------------------


class Sphere:
    """phi(x0) = a x0."""

    def __init__(self, a: float = 1.0):
        self.a = float(a)

    def phi(self, x0):
        return self.a * np.asarray(x0, dtype=np.float64)

    def jacobian(self, x0):
        x0 = np.asarray(x0)
        return np.broadcast_to(self.a * np.eye(3), x0.shape[:-1] + (3, 3)).copy()

    def describe(self):
        return {"shape": "sphere", "radius": self.a}


class Ellipsoid:
    """phi = beta o beta0^{-1} (Sec. 3.2): (x0, y0, z0) -> (a x0, b y0, c z0)."""

    def __init__(self, a: float, b: float, c: float):
        self.axes = np.array([a, b, c], dtype=np.float64)

    def phi(self, x0):
        return np.asarray(x0, dtype=np.float64) * self.axes

    def jacobian(self, x0):
        x0 = np.asarray(x0)
        return np.broadcast_to(np.diag(self.axes), x0.shape[:-1] + (3, 3)).copy()

    def describe(self):
        return {"shape": "ellipsoid", "axes": self.axes.tolist()}


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalized Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


class EvansFungRBC:
    """Biconcave red-blood-cell surface of radius 1 (Evans-Fung thickness law).

    phi(x0, y0, z0) = Q (x0, y0, z0 T(s) / 2),  s = x0^2 + y0^2,
    T(s) = C0 + C2 s + C4 s^2, so that on the unit sphere the height is
    +-(1/2) sqrt(1 - s) T(s): the Evans-Fung profile with unit radius. The
    map is a polynomial on R^3, hence a smooth diffeomorphism of S^2 onto the
    cell surface whenever T > 0 on [0, 1]. Q is a rotation.
    """

    C0, C2, C4 = 0.2072, 2.0026, -1.1228

    def __init__(self, rotation: np.ndarray | None = None):
        self.Q = np.eye(3) if rotation is None else np.asarray(rotation, dtype=np.float64)

    def _T(self, s):
        return self.C0 + self.C2 * s + self.C4 * s * s

    def _dT(self, s):
        return self.C2 + 2.0 * self.C4 * s

    def phi(self, x0):
        x0 = np.asarray(x0, dtype=np.float64)
        s = x0[..., 0] ** 2 + x0[..., 1] ** 2
        y = np.stack([x0[..., 0], x0[..., 1], 0.5 * x0[..., 2] * self._T(s)], axis=-1)
        return y @ self.Q.T

    def jacobian(self, x0):
        x0 = np.asarray(x0, dtype=np.float64)
        x, y, z = x0[..., 0], x0[..., 1], x0[..., 2]
        s = x * x + y * y
        J = np.zeros(x0.shape[:-1] + (3, 3))
        J[..., 0, 0] = 1.0
        J[..., 1, 1] = 1.0
        J[..., 2, 0] = z * x * self._dT(s)
        J[..., 2, 1] = z * y * self._dT(s)
        J[..., 2, 2] = 0.5 * self._T(s)
        return self.Q @ J

    def describe(self):
        return {"shape": "evans_fung_rbc", "radius": 1.0,
                "C0": self.C0, "C2": self.C2, "C4": self.C4,
                "rotation": self.Q.tolist()}


@dataclass
class Surface:
    """Quadrature nodes of one capsule surface on the m-th order grid."""

    m: int
    h: float
    patch: np.ndarray      # (N,) patch index 1..6
    j: np.ndarray          # (N,) u index 1..m-1
    k: np.ndarray          # (N,) v index 1..m-1
    x0: np.ndarray         # (N, 3) preimage on the unit sphere
    X: np.ndarray          # (N, 3) surface points
    W: np.ndarray          # (N,) area element |x_u x x_v|
    n: np.ndarray          # (N, 3) outward unit normal
    psi: np.ndarray        # (N,) partition-of-unity value of the owning patch
    w: np.ndarray          # (N,) quadrature weight psi * W * h^2
    shape: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_active(self) -> int:
        return int(np.count_nonzero(self.w))


@functools.lru_cache(maxsize=48)
def _sphere_grid(m: int):
    """Shape-independent part of a surface of order m: grid, preimages on the
    unit sphere, chart tangents and the POU value of the owning patch."""
    patch, j, k, u, v, x0 = patch_grid(m)
    du0 = np.empty_like(x0)
    dv0 = np.empty_like(x0)
    for i in range(1, 7):
        sel = patch == i
        du0[sel], dv0[sel] = chart_tangents(i, u[sel], v[sel])
    psi = pou_all(x0)[np.arange(len(patch)), patch - 1]
    for a in (patch, j, k, u, v, x0, du0, dv0, psi):
        a.setflags(write=False)
    return patch, j, k, u, v, x0, du0, dv0, psi


def make_surface(shape, m: int) -> Surface:
    """Build grid, POU and weights for surface map `shape` at order m."""
    patch, j, k, u, v, x0, du0, dv0, psi = _sphere_grid(m)
    h = np.pi / m
    J = shape.jacobian(x0)
    X = shape.phi(x0)
    xu = np.einsum("nab,nb->na", J, du0)
    xv = np.einsum("nab,nb->na", J, dv0)
    cr = np.cross(xu, xv)
    W = np.linalg.norm(cr, axis=-1)
    nrm = cr / W[:, None]
    w = psi * W * h * h
    return Surface(m=m, h=h, patch=patch, j=j, k=k, x0=x0, X=X, W=W, n=nrm,
                   psi=psi.copy(), w=w, shape=shape.describe())


def delta_star(surf: Surface, C: float = 1.0) -> np.ndarray:
    """Patch-dependent delta = C * delta* per node (Sec. 3.4, Eq. regparam).

    delta*_i is the largest, over the nodes of patch i, of the largest
    Euclidean distance from a node to its existing grid neighbours
    (offsets a, b in {-1, 0, 1}; neighbours outside 1..m-1 do not exist).
    """
    n = surf.m - 1
    X = surf.X.reshape(6, n, n, 3)
    best = np.zeros((6, n, n))
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a == 0 and b == 0:
                continue
            j0, j1 = max(0, a), n + min(0, a)
            k0, k1 = max(0, b), n + min(0, b)
            d = np.linalg.norm(X[:, j0:j1, k0:k1] - X[:, j0 - a:j1 - a, k0 - b:k1 - b], axis=-1)
            best[:, j0:j1, k0:k1] = np.maximum(best[:, j0:j1, k0:k1], d)
    per_patch = best.reshape(6, -1).max(axis=1)
    return C * per_patch[surf.patch - 1]
