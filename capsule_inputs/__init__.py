"""Seeded synthetic inputs for the regularized Stokes boundary sums.

This package builds the quadrature data that both the CUDA path and the CPU
oracle consume: the six-patch atlas of the unit sphere (Sec. 3.1, Eq.
param_maps), the partition of unity psi_i (Eq. pou0), the m-th order grid
(Sec. 3.2), the closed-form surface maps phi for the sphere, the ellipsoid
(Sec. 3.2, Eq. sphangles_ellip) and an Evans-Fung biconcave cell, the
smooth-quadrature weights w = psi * W * h_m^2 (Eq. smoothint), smooth random
densities, off-surface probe points and the patch-dependent regularization
parameter delta* (Eq. regparam).

It holds none of the layer-potential arithmetic: no kernel, no sum over
sources. Everything is numpy in float64 and deterministic for a given seed.
"""

from .geometry import (  # noqa: F401
    CHART_CENTERS,
    R0_POU,
    bump,
    chart,
    chart_tangents,
    patch_grid,
    pou_weight,
    Sphere,
    Ellipsoid,
    EvansFungRBC,
    random_rotation,
    Surface,
    make_surface,
    delta_star,
)
from .fields import real_sph_harm, sh_density, gaussian_noise  # noqa: F401
from .probes import exterior_probes  # noqa: F401
from .workloads import (  # noqa: F401
    Workload,
    sphere_noise_workload,
    rbc_workload,
    ellipsoid_hires_workload,
    serving_mix,
    grid_m_for_points_per_side,
)
