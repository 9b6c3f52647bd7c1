"""Off-surface probe points near a capsule surface.

A probe is x = phi(x0) + d * n(x0): x0 uniform on the unit sphere, n the
outward unit normal of the image surface (proportional to J^{-T} x0, the
cofactor transport of the sphere normal x0), and d log-uniform in
[dmin * h, dmax * h]. The paper has no off-surface evaluation; these probes
exercise the same regularized sums with targets that are not nodes.
"""

from __future__ import annotations

import numpy as np


def exterior_probes(shape, count: int, h: float, rng: np.random.Generator,
                    dmin: float = 0.1, dmax: float = 5.0, side: float = 1.0):
    """Return (points (count, 3), distances (count,)) on the side `side` (+1 out)."""
    x0 = rng.standard_normal((count, 3))
    x0 /= np.linalg.norm(x0, axis=1, keepdims=True)
    X = shape.phi(x0)
    J = shape.jacobian(x0)
    nrm = np.linalg.solve(np.swapaxes(J, -1, -2), x0[..., None])[..., 0]
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    d = h * np.exp(rng.uniform(np.log(dmin), np.log(dmax), size=count))
    return X + side * d[:, None] * nrm, d
