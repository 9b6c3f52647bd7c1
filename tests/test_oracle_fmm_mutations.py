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
from oracle import sl as oracle_sl

def _sl_fmm_variant(scale_far=True, gap=True, group=np.all):
    """sl_fmm with one of its decisions changed."""

    def sl_fmm(src, w, f, tgt, delta, mu, centers0, iters, p):
        src, tgt = np.asarray(src, np.float64), np.asarray(tgt, np.float64)
        w, f = np.asarray(w, np.float64), np.asarray(f, np.float64)
        delta = np.broadcast_to(np.asarray(delta, np.float64), (len(tgt),))
        act = w != 0.0
        src, w, f = src[act], w[act], f[act]
        k = len(centers0)
        _, labels = fmm.kmeans(src, centers0, iters)
        cen, a = fmm.boxes(src, labels, k)
        eq_pts, eq_den = fmm.equivalent_densities(src, w, f, labels, cen, a, p)
        u = np.zeros((len(tgt), 3))
        scale = 1.0 / (8.0 * np.pi * mu)
        for j in range(k):
            sel = labels == j
            if not np.any(sel):
                continue
            rel = np.abs(tgt - cen[j])
            far_t = rel.max(axis=1) >= fmm.R_CHECK * a[j]
            if gap:
                g = np.maximum(rel - a[j], 0.0)
                far_t &= (g * g).sum(axis=1) >= (fmm.RHO_FAR * delta) ** 2
            far = np.empty_like(far_t)
            for g0 in range(0, len(tgt), fmm.GROUP):
                far[g0:g0 + fmm.GROUP] = group(far_t[g0:g0 + fmm.GROUP])
            if np.any(far):
                s = scale if scale_far else 1.0
                u[far] += s * (fmm.stokeslet_matrix(tgt[far], eq_pts[j])
                               @ eq_den[j].ravel()).reshape(-1, 3)
            near = ~far
            if np.any(near):
                u[near] += oracle_sl(src[sel], w[sel], f[sel], tgt[near], delta[near], mu)
        return u

    return sl_fmm


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
    "far_field_without_1_over_8_pi_mu": {"sl_fmm": _sl_fmm_variant(scale_far=False)},
    "far_test_without_the_7_delta_gap": {"sl_fmm": _sl_fmm_variant(gap=False)},
    "group_far_if_any_target_is_far": {"sl_fmm": _sl_fmm_variant(group=np.any)},
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
