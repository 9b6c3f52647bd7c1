"""Plausible mistakes planted in the FMM oracle must fail its pins.

Each mutation replaces one step or constant of oracle/fmm.py (monkeypatched,
CPU only) and runs the pins of tests/test_oracle_fmm.py (all but the slow
convergence study) plus a lighter FMM-against-direct comparison (m = 16,
p = 6); at least one must fail.
"""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle
import test_oracle_fmm as pins
from oracle import fmm

def _neighbours_variant(centre_only=False, gap=True, gap_from_centre=False):
    """oracle/fmm.py's neighbour rule with one of its decisions changed."""

    def neighbours(lo, hi, delta_i, cen, a):
        if centre_only:   # the box's centre instead of the whole box
            lo = hi = 0.5 * (lo + hi)
        outside_check = np.any((lo[None] > cen + fmm.R_CHECK * a[:, None]) |
                               (hi[None] < cen - fmm.R_CHECK * a[:, None]), axis=1)
        half = 0.0 if gap_from_centre else a[:, None]
        g = np.maximum(np.maximum(lo[None] - (cen + half), (cen - half) - hi[None]), 0.0)
        gap2 = (g * g).sum(axis=1)
        far = outside_check
        if gap:
            far = far & (gap2 >= (fmm.RHO_FAR * delta_i) ** 2)
        return ~far

    return neighbours


def _plan_with_smallest_delta(src, w, tgt, delta, centers0, iters):
    """plan() with the smallest delta of a target box instead of the largest."""
    delta = np.broadcast_to(np.asarray(delta, np.float64), (len(tgt),))
    pl = _PLAN(src, w, tgt, delta, centers0, iters)
    tgt = np.asarray(tgt, np.float64)
    for i in range(len(pl["cen"])):
        ti = np.flatnonzero(pl["tlab"] == i)
        if len(ti):
            T = tgt[ti]
            pl["near"][i] = fmm.neighbours(T.min(0), T.max(0), float(delta[ti].min()), pl["cen"],
                                           pl["a"])
    return pl


def _far_field_without_scale(T, E, phi):
    return 8.0 * np.pi * _FAR_FIELD(T, E, phi)   # pins use mu = 1


_PLAN = fmm.plan
_FAR_FIELD = fmm.far_field


def component_major_columns(targets, sources):
    """The (3 nt, 3 ns) matrix with its columns ordered component-major
    (b ns + s) while the densities it multiplies are raveled source-major
    (3 s + b)."""
    d = targets[:, None, :] - sources[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    G = np.eye(3)[None, None] / r[..., None, None] + d[..., :, None] * d[..., None, :] / (
        r ** 3)[..., None, None]
    return G.transpose(0, 2, 3, 1).reshape(3 * len(targets), 3 * len(sources))


def kmeans_without_updates(points, centers0, iters):
    """Lloyd iterations whose centres never move."""
    c = np.array(centers0, dtype=np.float64, copy=True)
    d = points[:, None, :] - c[None, :, :]
    return c, np.argmin((d * d).sum(-1), axis=1)


MUTATIONS = {
    "far_field_without_1_over_8_pi_mu": {"far_field": _far_field_without_scale},
    "far_test_without_the_7_delta_gap": {"neighbours": _neighbours_variant(gap=False)},
    "far_if_the_box_centre_is_outside_the_check_cube":
        {"neighbours": _neighbours_variant(centre_only=True)},
    "gap_from_the_cluster_centre": {"neighbours": _neighbours_variant(gap_from_centre=True)},
    "smallest_delta_of_the_box": {"plan": _plan_with_smallest_delta},
    "equivalent_and_check_radii_swapped": {"R_EQUIV": fmm.R_CHECK, "R_CHECK": fmm.R_EQUIV},
    "stokeslet_columns_component_major": {"stokeslet_matrix": component_major_columns},
    "kmeans_without_updates": {"kmeans": kmeans_without_updates},
}


def fmm_matches_direct_at_p6():
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 16)
    f = ci.sh_density(s.x0, np.random.default_rng(3), lmax=6)
    act = np.flatnonzero(s.w)
    c0 = s.X[act[:: len(act) // 20][:20]]
    tgt = s.X[::5]
    ref = oracle.sl(s.X, s.w, f, tgt, 0.02)
    u = fmm.sl_fmm(s.X, s.w, f, tgt, 0.02, 1.0, c0, 8, 6)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-5


PINS = [
    pins.test_neighbour_rule_is_box_against_box,
    pins.test_cube_surface_grid,
    pins.test_kmeans_invariants,
    pins.test_equivalent_sources_reproduce_far_potential,
    pins.test_all_near_is_the_direct_sum,
    pins.test_clusters_within_seven_delta_are_summed_directly,
    fmm_matches_direct_at_p6,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_fails_a_pin(name, monkeypatch):
    for attr, repl in MUTATIONS[name].items():
        monkeypatch.setattr(fmm, attr, repl)
    failed = 0
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except (AssertionError, np.linalg.LinAlgError):
            failed += 1
    assert failed >= 1, f"mutation {name} passed every pin"


def test_unmutated_oracle_passes_the_same_pins():
    for pin in PINS:
        pin()
