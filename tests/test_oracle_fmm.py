"""Pins of the single-level FMM oracle (oracle/fmm.py, Sec. 5):

* the cube surface grid has 6p^2 - 12p + 8 points, all on the surface;
* k-means returns the nearest-centre assignment of its final centres, and
  a cluster's centre is the mean of its points at a fixed point of Lloyd;
* one cluster's equivalent sources reproduce its plain-Stokeslet potential
  outside the check cube, with an error that falls quickly with p;
* with every cluster near (huge delta), the FMM is the direct sum;
* on an ellipsoid, the FMM approaches the direct regularized sum as p grows;
* the plain Stokeslet of the far field has its closed form;
* the neighbour rule is box against box (Sec. 5, step 3), checked against
  an independent computation of box distances, and every far (box, cluster)
  pair is valid for each of its targets: outside the check cube and at least
  7 delta (the target's own) from the cluster cube.
"""

import numpy as np

import capsule_inputs as ci
import oracle
from oracle import fmm


def test_cube_surface_grid():
    for p in (3, 4, 5, 6):
        pts = fmm.cube_surface(p)
        assert len(pts) == 6 * p * p - 12 * p + 8
        assert np.allclose(np.abs(pts).max(axis=1), 1.0)
        assert len(np.unique(pts.round(12), axis=0)) == len(pts)


def test_kmeans_invariants():
    rng = np.random.default_rng(0)
    pts = rng.standard_normal((500, 3))
    c, lab = fmm.kmeans(pts, pts[:8], 50)
    d2 = ((pts[:, None] - c[None]) ** 2).sum(-1)
    assert np.array_equal(lab, np.argmin(d2, axis=1))
    for j in range(8):
        assert np.allclose(c[j], pts[lab == j].mean(axis=0), atol=1e-12)


def test_equivalent_sources_reproduce_far_potential():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.5, 0.5, (300, 3))
    w = rng.uniform(0.5, 1.5, 300)
    f = rng.standard_normal((300, 3))
    lab = np.zeros(300, dtype=int)
    cen, a = fmm.boxes(pts, lab, 1)
    d = rng.standard_normal((200, 3))
    far = cen[0] + 3.0 * a[0] * d / np.abs(d).max(axis=1, keepdims=True)   # on the 3a cube
    exact = fmm.stokeslet_matrix(far, pts) @ (w[:, None] * f).ravel()
    errs = []
    for p in (4, 6, 8):
        E, phi = fmm.equivalent_densities(pts, w, f, lab, cen, a, p)
        approx = fmm.stokeslet_matrix(far, E[0]) @ phi[0].ravel()
        errs.append(np.abs(approx - exact).max() / np.abs(exact).max())
    assert errs[-1] < 1e-5 and errs[-1] < errs[0] / 100, errs


def test_all_near_is_the_direct_sum():
    s = ci.make_surface(ci.Sphere(1.0), 9)
    f = ci.sh_density(s.x0, np.random.default_rng(2), lmax=4)
    c0 = s.X[s.w != 0][::40]
    u = fmm.sl_fmm(s.X, s.w, f, s.X, 10.0, 1.3, c0, 5, 4)
    ref = oracle.sl(s.X, s.w, f, s.X, 10.0, 1.3)
    assert np.allclose(u, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_fmm_converges_to_the_direct_sum():
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 24)
    f = ci.sh_density(s.x0, np.random.default_rng(3), lmax=6)
    act = np.flatnonzero(s.w)
    c0 = s.X[act[:: len(act) // 30][:30]]
    tgt = s.X[::7]
    delta = 0.02   # small enough that most clusters are far (7 delta from their cube)
    ref = oracle.sl(s.X, s.w, f, tgt, delta)
    errs = []
    for p in (4, 6, 8):
        u = fmm.sl_fmm(s.X, s.w, f, tgt, delta, 1.0, c0, 8, p)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[2] < 1e-5 and errs[2] < errs[1] < errs[0], errs


def test_clusters_within_seven_delta_are_summed_directly():
    """delta = 0.5 on an ellipsoid with 20 clusters: 41% of the (target,
    cluster) pairs lie outside the check cube, but all lie within 7 delta of
    the cluster cube, where the regularized kernel differs from the plain one;
    so every cluster is summed directly and the FMM is the direct sum."""
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 16)
    f = ci.sh_density(s.x0, np.random.default_rng(4), lmax=6)
    act = np.flatnonzero(s.w)
    c0 = s.X[act[:: len(act) // 20][:20]]
    tgt = s.X[::5]
    _, lab = fmm.kmeans(s.X[act], c0, 8)
    cen, a = fmm.boxes(s.X[act], lab, 20)
    outside = np.mean([(np.abs(tgt - cen[j]).max(axis=1) >= fmm.R_CHECK * a[j]).mean()
                       for j in range(20)])
    assert outside > 0.3
    u = fmm.sl_fmm(s.X, s.w, f, tgt, 0.5, 1.0, c0, 8, 6)
    ref = oracle.sl(s.X, s.w, f, tgt, 0.5)
    assert np.allclose(u, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_plain_stokeslet_closed_form():
    """One source g = (1, 2, -1) at the origin, target at (0, 0, 10) and at
    (3, 4, 0): v = g / r + (g . d) d / r^3 (Sec. 2.2), written out."""
    g = np.array([[1.0, 2.0, -1.0]])
    v = oracle.plain_stokeslet(np.zeros((1, 3)), g, [[0.0, 0.0, 10.0], [3.0, 4.0, 0.0]])
    assert np.allclose(v[0], [0.1, 0.2, -0.1 - 0.1], rtol=1e-15)
    assert np.allclose(v[1], [0.2 + 11 * 3 / 125, 0.4 + 11 * 4 / 125, -0.2], rtol=1e-15)
    # and the regularized sum far from the sources (rho >= 100) is the plain one
    rng = np.random.default_rng(6)
    X = rng.uniform(-0.5, 0.5, (40, 3))
    w = rng.uniform(0.5, 1.0, 40)
    f = rng.standard_normal((40, 3))
    Y = rng.uniform(2.0, 3.0, (10, 3))
    ref = oracle.sl(X, w, f, Y, 0.01, 1.0) * 8 * np.pi
    assert np.allclose(oracle.plain_stokeslet(X, w[:, None] * f, Y), ref, rtol=1e-13)


def fmm_case(m=16, k=20, n_probes=300, seed=9):
    """Ellipsoid nodes plus near exterior probes, one delta per target."""
    rng = np.random.default_rng(seed)
    shape = ci.Ellipsoid(1.0, 0.8, 0.5)
    s = ci.make_surface(shape, m)
    probes, _ = ci.exterior_probes(shape, n_probes, s.h, rng)
    tgt = np.concatenate([s.X[::2], probes])
    delta = rng.uniform(0.05, 0.15, len(tgt))
    act = np.flatnonzero(s.w)
    c0 = s.X[act[:: len(act) // k][:k]]
    return s, tgt, delta, c0


def test_neighbour_rule_is_box_against_box():
    s, tgt, delta, c0 = fmm_case()
    pl = fmm.plan(s.X, s.w, tgt, delta, c0, 8)
    cen, a, tlab, near, cent = pl["cen"], pl["a"], pl["tlab"], pl["near"], pl["centers"]
    # targets join their nearest final centre
    dist = np.linalg.norm(tgt[:, None] - cent[None], axis=-1)
    assert np.array_equal(tlab, np.argmin(dist, axis=1))
    counts = np.bincount(pl["labels"], minlength=len(cen))
    n_far = 0
    for i in np.unique(tlab):
        ti = np.flatnonzero(tlab == i)
        T = tgt[ti]
        bc, bh = 0.5 * (T.min(0) + T.max(0)), 0.5 * (T.max(0) - T.min(0))
        for j in np.flatnonzero(counts):
            sep = np.abs(bc - cen[j]) - bh            # per axis, box centre to box edge
            outside_check = np.any(sep > fmm.R_CHECK * a[j])
            gap = np.linalg.norm(np.maximum(sep - a[j], 0.0))
            far = outside_check and gap >= fmm.RHO_FAR * delta[ti].max()
            assert near[i, j] == (not far), (i, j)
            if far:
                n_far += 1
                # valid for every target of the box, with its own delta
                rel = np.abs(T - cen[j])
                assert np.all(rel.max(axis=1) > fmm.R_CHECK * a[j])
                g = np.linalg.norm(np.maximum(rel - a[j], 0.0), axis=1)
                assert np.all(g >= fmm.RHO_FAR * delta[ti])
    assert n_far > 0 and not near.all()
