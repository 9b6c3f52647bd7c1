"""Plausible mistakes planted in the upsampling oracle must fail its pins.

Each mutation replaces one step of oracle/upsample.py (monkeypatched, CPU
only) and runs the pins of tests/test_oracle_upsample.py that cover it (all
but the slow m = 48 table comparison); at least one must fail.
"""

import numpy as np
import pytest

import capsule_inputs as ci
import test_oracle_upsample as pins
from oracle import sl as oracle_sl
from oracle import upsample as up

_orig_upsample = up.upsample
_orig_fine_pou = up.fine_pou
_orig_fine_delta = up.fine_delta_star


def _sl_upsampled_with(weights):
    """sl_upsampled with the fine weights given by weights(m, q, Wu, hu)."""

    def sl_upsampled(m, X, W, f, mu=1.0, q=up.FACTOR, targets=None):
        Xu, Wu, Fu = up.upsample(m, X, q), up.upsample(m, W, q), up.upsample(m, f, q)
        hu = np.pi / (q * m)
        wu = weights(m, q, Wu, hu)
        d_patch = up.fine_delta_star(m, Xu, q).reshape(6, -1)[:, 0]
        d_tgt = np.repeat(d_patch, (m - 1) ** 2)
        idx = np.arange(X.shape[0]) if targets is None else np.asarray(targets)
        return oracle_sl(Xu, wu, Fu, X[idx], d_tgt[idx], mu)

    return sl_upsampled


# the coarse spacing pi / m in the fine weights (16x too large)
coarse_spacing_in_weights = _sl_upsampled_with(
    lambda m, q, Wu, hu: up.fine_pou(m, q) * Wu * (np.pi / m) ** 2)
# the fine area element left out: psi_u h_u^2
area_element_not_upsampled = _sl_upsampled_with(lambda m, q, Wu, hu: up.fine_pou(m, q) * hu * hu)


def pou_of_the_next_patch(m, q=up.FACTOR):
    """psi of patch p + 1 (cyclically) at the fine nodes of patch p."""
    from capsule_inputs.geometry import chart, pou_all
    _, u, v = up.fine_grid(m, q)
    return np.concatenate([pou_all(chart(p, u, v))[:, p % 6] for p in range(1, 7)])


def coarse_delta_for_targets(m, Xu, q=up.FACTOR, C=1.0):
    """delta* of the coarse grid (the coarse nodes are fine nodes 4j, 4k)."""
    nf, n = q * m - 1, m - 1
    Xc = Xu.reshape(6, nf, nf, 3)[:, q - 1::q, q - 1::q][:, :n, :n].reshape(-1, 3)
    surf = ci.make_surface(ci.Sphere(1.0), m)
    surf.X = Xc
    d = ci.delta_star(surf, C).reshape(6, -1)[:, :1]
    return np.repeat(d, nf * nf, axis=1).ravel()


def linear_interpolation(m, G, q=up.FACTOR):
    """Bilinear instead of cubic-spline interpolation on each patch."""
    from scipy.interpolate import RegularGridInterpolator
    G = np.asarray(G, dtype=np.float64)
    flat = G.reshape(G.shape[0], -1)
    Gp = flat.reshape(6, m - 1, m - 1, -1)
    nodes = np.arange(1, m) * (np.pi / m)
    _, u, v = up.fine_grid(m, q)
    pts = np.stack([u, v], axis=1)
    out = np.concatenate([
        RegularGridInterpolator((nodes, nodes), Gp[p], method="linear", bounds_error=False,
                                fill_value=None)(pts) for p in range(6)], axis=0)
    return out.reshape((out.shape[0],) + G.shape[1:])


MUTATIONS = {
    "coarse_spacing_in_weights": ("sl_upsampled", coarse_spacing_in_weights),
    "area_element_not_upsampled": ("sl_upsampled", area_element_not_upsampled),
    "pou_of_the_next_patch": ("fine_pou", pou_of_the_next_patch),
    "coarse_delta_for_targets": ("fine_delta_star", coarse_delta_for_targets),
    "linear_interpolation": ("upsample", linear_interpolation),
}

PINS = [
    pins.test_upsampling_is_exact_on_bicubics_and_interpolates,
    pins.test_fine_weights_integrate_the_area,
    pins.test_uniform_traction_on_a_sphere_improves_with_upsampling,
    pins.test_coarse_nodes_match_a_finer_upsampled_solution,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_fails_a_pin(name, monkeypatch):
    attr, repl = MUTATIONS[name]
    monkeypatch.setattr(up, attr, repl)
    failed = 0
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, f"mutation {name} passed every pin"


def test_unmutated_oracle_passes_the_same_pins():
    for pin in PINS:
        pin()
