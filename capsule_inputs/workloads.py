"""Named synthetic workloads (seeded) for tests and benchmarks.

Seeds follow seed = 1000 * workload_index + k. "n x n points per patch"
means the m-th order grid with m = n + 1, since a patch holds (m-1)^2 nodes
(Sec. 3.2). "delta = C h" means the global delta = C pi / m (Appendix,
Table sing_int_delta, columns delta = C h_m).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .fields import gaussian_noise, sh_density
from .geometry import (Ellipsoid, EvansFungRBC, Sphere, Surface, make_surface,
                       random_rotation)
from .probes import exterior_probes


def grid_m_for_points_per_side(n: int) -> int:
    """m such that one patch has n x n nodes: (m - 1)^2 = n^2."""
    return int(n) + 1


@dataclass
class Workload:
    """Sources (nodes of one surface), densities, targets and delta."""

    name: str
    surface: Surface
    f: np.ndarray                 # (N, 3) single-layer density (traction)
    targets: np.ndarray           # (M, 3)
    delta: np.ndarray             # (M,) or (1,)
    mu: float = 1.0
    q: np.ndarray | None = None   # (N, 3) double-layer density
    n_on_surface: int = 0         # targets[:n_on_surface] are the nodes themselves
    meta: dict = field(default_factory=dict)

    @property
    def sources(self):
        s = self.surface
        return s.X, s.w, s.n

    def interactions(self) -> int:
        """M_targets x N_s (sources with nonzero weight)."""
        return int(self.targets.shape[0]) * self.surface.n_active


def sphere_noise_workload(m: int = 19, seed: int = 1000, delta_factor: float = 2.0,
                          sigma: float = 0.1) -> Workload:
    """Unit sphere, 18x18 nodes per patch (m = 19, N = 1944); f = e_x + N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    surf = make_surface(Sphere(1.0), m)
    f = np.zeros((surf.N, 3))
    f[:, 0] = 1.0
    f += gaussian_noise(surf.N, sigma, rng)
    delta = np.array([delta_factor * surf.h])
    return Workload(name=f"sphere m={m} N={surf.N} delta={delta_factor}h", surface=surf, f=f,
                    targets=surf.X.copy(), delta=delta, mu=1.0, n_on_surface=surf.N,
                    meta={"seed": seed, "delta_factor": delta_factor})


def rbc_workload(m: int = 65, seed: int = 2000, delta_factor: float = 2.0) -> Workload:
    """Rotated Evans-Fung cell, 64x64 per patch (m = 65, N = 24,576); SH densities."""
    rng = np.random.default_rng(seed)
    shape = EvansFungRBC(random_rotation(rng))
    surf = make_surface(shape, m)
    f = sh_density(surf.x0, rng, lmax=8)
    q = sh_density(surf.x0, rng, lmax=8)
    delta = np.array([delta_factor * surf.h])
    return Workload(name=f"rbc m={m} N={surf.N} delta={delta_factor}h", surface=surf, f=f,
                    q=q, targets=surf.X.copy(), delta=delta, mu=1.0, n_on_surface=surf.N,
                    meta={"seed": seed, "delta_factor": delta_factor})


def ellipsoid_hires_workload(m: int = 257, seed: int = 3000, delta_factor: float = 2.0,
                             n_probes: int = 100_000, axes=(1.0, 0.8, 0.5)) -> Workload:
    """Ellipsoid (1, 0.8, 0.5), 256x256 per patch (m = 257, N = 393,216).

    Targets are the N nodes followed by n_probes exterior probes at distances
    log-uniform in [0.1 h, 5 h]; delta = delta_factor * h for all targets.
    """
    rng = np.random.default_rng(seed)
    shape = Ellipsoid(*axes)
    surf = make_surface(shape, m)
    f = sh_density(surf.x0, rng, lmax=8)
    if n_probes > 0:
        probes, _ = exterior_probes(shape, n_probes, surf.h, rng)
        targets = np.concatenate([surf.X, probes], axis=0)
    else:
        targets = surf.X.copy()
    delta = np.array([delta_factor * surf.h])
    return Workload(name=f"ellipsoid{tuple(axes)} m={m} N={surf.N} delta={delta_factor}h "
                         f"+{n_probes} probes",
                    surface=surf, f=f, targets=targets, delta=delta, mu=1.0,
                    n_on_surface=surf.N,
                    meta={"seed": seed, "delta_factor": delta_factor, "n_probes": n_probes})


def serving_mix(n_requests: int = 1000, seed: int = 4000, n_min: int = 1536,
                n_max: int = 98_304, rate_hz: float = 100.0):
    """Request specs for the serving mix (shapes are built on demand).

    Each request: shape 50/50 ellipsoid (axes sorted, U[0.5, 1]) or rotated
    cell; N log-uniform in [n_min, n_max] rounded to N = 6 n^2; Poisson
    arrivals at rate_hz; density seed per request.
    """
    rng = np.random.default_rng(seed)
    specs = []
    t = 0.0
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        N = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        n = int(round(np.sqrt(N / 6.0)))
        n = max(2, n)
        if rng.uniform() < 0.5:
            axes = np.sort(rng.uniform(0.5, 1.0, size=3))[::-1]
            shape = ("ellipsoid", tuple(float(a) for a in axes))
        else:
            shape = ("rbc", tuple(float(x) for x in rng.standard_normal(4)))
        specs.append({"id": r, "arrival_s": t, "m": n + 1, "shape": shape,
                      "seed": seed + 1 + r})
    return specs


def build_request(spec, delta_factor: float = 2.0):
    """Surface, density and delta for one serving request spec."""
    kind, params = spec["shape"]
    if kind == "ellipsoid":
        shape = Ellipsoid(*params)
    else:
        q = np.asarray(params, dtype=np.float64)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        Q = np.array([
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ])
        shape = EvansFungRBC(Q)
    surf = make_surface(shape, spec["m"])
    rng = np.random.default_rng(spec["seed"])
    f = sh_density(surf.x0, rng, lmax=8)
    return surf, f, delta_factor * surf.h
