"""Pins for the seeded input generator (atlas, POU, grid, weights, normals)."""

import numpy as np
import pytest

import capsule_inputs as ci
from conftest import read_golden


def test_charts_cover_hemispheres_and_centres():
    # Sec. 3.1, Eq. param_maps: six hemispherical patches centred on the +-axes.
    centres = {tuple(np.round(c).astype(int)) for c in ci.CHART_CENTERS}
    assert centres == {(0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0), (0, 0, 1), (0, 0, -1)}
    u = np.linspace(0.05, np.pi - 0.05, 13)
    U, V = np.meshgrid(u, u, indexing="ij")
    for i in range(1, 7):
        x = ci.chart(i, U, V)
        assert np.allclose(np.linalg.norm(x, axis=-1), 1.0)
        # every chart point lies in the open hemisphere around its centre
        assert np.all(x @ ci.CHART_CENTERS[i - 1] > 0)


def test_chart_tangents_match_finite_differences_and_orientation():
    rng = np.random.default_rng(1)
    u = rng.uniform(0.2, np.pi - 0.2, 50)
    v = rng.uniform(0.2, np.pi - 0.2, 50)
    eps = 1e-6
    for i in range(1, 7):
        du, dv = ci.chart_tangents(i, u, v)
        fdu = (ci.chart(i, u + eps, v) - ci.chart(i, u - eps, v)) / (2 * eps)
        fdv = (ci.chart(i, u, v + eps) - ci.chart(i, u, v - eps)) / (2 * eps)
        assert np.abs(du - fdu).max() < 1e-8
        assert np.abs(dv - fdv).max() < 1e-8
        # |x_u x x_v| = sin u and the cross product points outward for all charts
        cr = np.cross(du, dv)
        assert np.allclose(np.linalg.norm(cr, axis=-1), np.sin(u))
        assert np.all(np.sum(cr * ci.chart(i, u, v), axis=-1) > 0)


def test_bump_values():
    # b(0) = 1, b -> 0 as |r| -> 1, zero outside (Sec. 3.1).
    assert ci.bump(0.0) == 1.0
    assert ci.bump(0.999999) < 1e-100
    assert ci.bump(1.0) == 0.0 and ci.bump(1.5) == 0.0
    assert ci.bump(-0.3) == ci.bump(0.3)
    r = np.linspace(0, 0.99, 100)
    assert np.all(np.diff(ci.bump(r)) <= 0)


def test_partition_of_unity_sums_to_one_and_support():
    rng = np.random.default_rng(2)
    x0 = rng.standard_normal((5000, 3))
    x0 /= np.linalg.norm(x0, axis=1, keepdims=True)
    psi = ci.geometry.pou_all(x0)
    assert np.allclose(psi.sum(axis=1), 1.0, atol=1e-14)
    # supp psi_i is the cap of great-circle radius r0 = 5 pi / 12 around its centre
    for i in range(6):
        d = ci.geometry.great_circle(x0, ci.CHART_CENTERS[i])
        assert np.all(psi[d >= ci.R0_POU, i] == 0.0)
        assert np.all(psi[d < ci.R0_POU - 0.05, i] > 0.0)  # b underflows within ~1e-3 rad of the edge


@pytest.mark.parametrize("row", read_golden("grid_sizes.txt"))
def test_grid_sizes_match_paper_table(row):
    m, N, Nup = map(int, row)
    assert ci.patch_grid(m)[0].shape[0] == N
    # the printed upsampled sizes are 16 N: 4x the nodes per side (the m = 48
    # row's N_up belongs to m = 64, see the fixture's header)
    if m == 48:
        assert Nup == 16 * ci.patch_grid(64)[0].shape[0]
    else:
        assert 16 * N == Nup == 6 * (4 * (m - 1)) ** 2


def test_sphere_area_converges_superalgebraically():
    errs = []
    for m in (17, 33, 65):
        s = ci.make_surface(ci.Sphere(1.0), m)
        errs.append(abs(s.w.sum() / (4 * np.pi) - 1))
    assert errs[-1] < 1e-7
    assert errs[0] / errs[1] > 50 and errs[1] / errs[2] > 50


@pytest.mark.parametrize("row", read_golden("ellipsoid_area_volume.txt"))
def test_ellipsoid_area_volume_within_paper_table(row):
    m, N = int(row[0]), int(row[1])
    epsA, epsV = float(row[2]), float(row[3])
    s = ci.make_surface(ci.Ellipsoid(0.6, 1.0, 1.0), m)
    assert s.N == N
    e = 0.8  # oblate spheroid, equatorial radius 1, polar semi-axis 0.6
    A = 2 * np.pi * (1 + (1 - e * e) / e * np.arctanh(e))
    V = 4.0 / 3.0 * np.pi * 0.6
    # volume by the divergence theorem with M = (x, 0, 0) (Sec. 4.1, footnote)
    assert abs(s.w.sum() / A - 1) <= epsA
    assert abs(np.sum(s.w * s.X[:, 0] * s.n[:, 0]) / V - 1) <= epsV


def test_ellipsoid_area_against_legendre_closed_form():
    from scipy.special import ellipeinc, ellipkinc
    a, b, c = 1.0, 0.8, 0.5
    phi = np.arccos(c / a)
    k2 = a * a * (b * b - c * c) / (b * b * (a * a - c * c))
    A = 2 * np.pi * c * c + 2 * np.pi * a * b / np.sin(phi) * (
        ellipeinc(phi, k2) * np.sin(phi) ** 2 + ellipkinc(phi, k2) * np.cos(phi) ** 2)
    s = ci.make_surface(ci.Ellipsoid(a, b, c), 65)
    assert abs(s.w.sum() / A - 1) < 1e-6


def test_normals_are_outward_unit_and_match_implicit_gradient():
    axes = np.array([1.0, 0.8, 0.5])
    s = ci.make_surface(ci.Ellipsoid(*axes), 33)
    g = s.X / axes ** 2
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    assert np.abs(s.n - g).max() < 1e-13
    assert np.all(np.sum(s.n * s.X, axis=1) > 0)


def test_rbc_volume_area_against_axisymmetric_quadrature():
    from scipy.integrate import quad
    shape = ci.EvansFungRBC(ci.random_rotation(np.random.default_rng(3)))
    s = ci.make_surface(shape, 65)
    C0, C2, C4 = shape.C0, shape.C2, shape.C4

    def height(r):  # half-thickness of the cell at radius r
        q = r * r
        return 0.5 * np.sqrt(max(0.0, 1.0 - q)) * (C0 + C2 * q + C4 * q * q)

    V = 2 * quad(lambda r: 2 * np.pi * r * height(r), 0, 1, limit=200)[0]
    Vq = np.sum(s.w * np.sum(s.X * s.n, axis=1)) / 3.0
    assert abs(Vq / V - 1) < 1e-6
    # the rotation leaves the weights (areas) unchanged
    s0 = ci.make_surface(ci.EvansFungRBC(), 65)
    assert np.allclose(s.w, s0.w, rtol=1e-12, atol=1e-15)


def test_delta_star_on_sphere_is_sqrt2_h():
    # Eq. regparam: the largest neighbour distance is the diagonal at the
    # patch centre, 2 sin(h/sqrt 2 ...) ~ sqrt(2) h for small h.
    for m in (19, 65):
        s = ci.make_surface(ci.Sphere(1.0), m)
        d = ci.delta_star(s)
        assert np.allclose(d, d[0])
        assert abs(d[0] / s.h - np.sqrt(2)) < 0.01


def test_real_sph_harm_orthonormal():
    # Gauss-Legendre in cos(theta) x trapezoid in phi integrates degree <= 16 exactly
    xs, ws = np.polynomial.legendre.leggauss(20)
    ph = 2 * np.pi * np.arange(40) / 40
    Z, P = np.meshgrid(xs, ph, indexing="ij")
    W = (ws[:, None] * np.full_like(P, 2 * np.pi / 40)).ravel()
    st = np.sqrt(1 - Z ** 2)
    x0 = np.stack([st * np.cos(P), st * np.sin(P), Z], -1).reshape(-1, 3)
    Y = ci.real_sph_harm(8, x0)
    G = (Y * W[:, None]).T @ Y
    assert np.abs(G - np.eye(81)).max() < 1e-12


def test_workloads_are_deterministic_and_sized():
    w1 = ci.sphere_noise_workload()
    w2 = ci.sphere_noise_workload()
    assert w1.surface.N == 1944 and w1.surface.n_active == 1344
    assert np.array_equal(w1.f, w2.f)
    r = ci.rbc_workload(m=17)
    assert r.q is not None and r.surface.N == 6 * 16 ** 2
    e = ci.ellipsoid_hires_workload(m=33, n_probes=500)
    assert e.targets.shape[0] == e.surface.N + 500
    # probes lie outside the ellipsoid, between 0.1 h and 5 h from it
    P = e.targets[e.surface.N:]
    lev = np.sum((P / np.array([1.0, 0.8, 0.5])) ** 2, axis=1)
    assert np.all(lev > 1.0)


def test_probe_distances():
    rng = np.random.default_rng(5)
    shape = ci.Sphere(1.0)
    P, d = ci.exterior_probes(shape, 2000, 0.01, rng)
    assert np.allclose(np.linalg.norm(P, axis=1) - 1.0, d)
    assert d.min() >= 0.1 * 0.01 - 1e-15 and d.max() <= 5 * 0.01 + 1e-15


def test_serving_mix_sizes():
    specs = ci.serving_mix(200)
    Ns = [6 * (s["m"] - 1) ** 2 for s in specs]
    assert min(Ns) >= 1536 and max(Ns) <= 98_304
    t = [s["arrival_s"] for s in specs]
    assert np.all(np.diff(t) > 0)
