"""Pins of the membrane oracle (oracle/membrane.py) to facts independent of it.

* transition maps: round trip, the Appendix's printed formulas, and their
  Jacobians against central differences of the maps themselves;
* spline and stencil: exact on cubics (spline, incl. its end pieces) and on
  polynomials of degree <= 6 (7-point stencil);
* the derivative scheme against closed-form normals, curvatures and a surface
  divergence on the sphere and the ellipsoid (0.6, 1, 1): at or below the
  errors printed in Sec. 4.2 / Appendix (golden derivative_errors.txt), with
  fourth-order convergence;
* the Skalak force (Eqs. tensor, intf): zero at the stress-free reference,
  the closed form -2T/a n of a uniformly dilated sphere, and virtual work
  int f . v dA = -dE/de against the Skalak strain energy
  W_s = Es/4 (I1^2/2 + I1 - I2) + ED/8 I2^2, whose Cauchy tension is Eq. tensor;
* area and volume of the ellipsoid against the closed forms.
"""

import numpy as np
import pytest

import capsule_inputs as ci
from capsule_inputs.geometry import chart
from conftest import read_golden
from oracle import membrane as mb

ES, ED = 2.0, 20.0


def golden():
    out = {}
    for shape, m, _, en, eH, eK, ed in read_golden("derivative_errors.txt"):
        out[(shape, int(m))] = tuple(float(x) for x in (en, eH, eK, ed))
    return out


def rel_inf(a, b):
    if not np.all(np.isfinite(a)):
        return float("inf")
    return float(np.abs(a - b).max() / np.abs(b).max())


# ---- transition maps --------------------------------------------------------
def test_inverse_chart_round_trip():
    u, v = np.meshgrid(np.linspace(0.05, np.pi - 0.05, 23), np.linspace(0.05, np.pi - 0.05, 19))
    for p in range(1, 7):
        uu, vv = mb.inverse_chart(p, chart(p, u, v))
        assert np.allclose(uu, u, atol=1e-13) and np.allclose(vv, v, atol=1e-13)


def _printed_transitions():
    """The transition maps as printed in the Appendix, except tau_56 / tau_65
    (printed as (pi - u, v)) and tau_63 / tau_64 (sign of cos u), which are
    checked against the chart composition below."""
    s, c, acos, sq = np.sin, np.cos, np.arccos, np.sqrt

    def t5x(su_sv_sign, cos_num):  # helper for the acos/acos family
        return lambda u, v: (acos(su_sv_sign(u, v)), acos(cos_num(u, v)))

    A = lambda u, v: sq(s(u) ** 2 * c(v) ** 2 + c(u) ** 2)
    B = lambda u, v: sq(s(u) ** 2 * s(v) ** 2 + c(u) ** 2)
    return {
        (1, 2): lambda u, v: (u, np.pi + v), (1, 3): lambda u, v: (u, np.pi / 2 + v),
        (1, 4): lambda u, v: (u, v - np.pi / 2),
        (1, 5): t5x(lambda u, v: -s(u) * s(v), lambda u, v: s(u) * c(v) / A(u, v)),
        (1, 6): t5x(lambda u, v: s(u) * s(v), lambda u, v: s(u) * c(v) / A(u, v)),
        (2, 1): lambda u, v: (u, np.pi + v), (2, 3): lambda u, v: (u, v - np.pi / 2),
        (2, 4): lambda u, v: (u, v + np.pi / 2),
        (2, 5): t5x(lambda u, v: s(u) * s(v), lambda u, v: -s(u) * c(v) / A(u, v)),
        (2, 6): t5x(lambda u, v: -s(u) * s(v), lambda u, v: -s(u) * c(v) / A(u, v)),
        (3, 1): lambda u, v: (u, v - np.pi / 2), (3, 2): lambda u, v: (u, v + np.pi / 2),
        (3, 4): lambda u, v: (u, v + np.pi),
        (3, 5): t5x(lambda u, v: s(u) * c(v), lambda u, v: s(u) * s(v) / B(u, v)),
        (3, 6): t5x(lambda u, v: -s(u) * c(v), lambda u, v: s(u) * s(v) / B(u, v)),
        (4, 1): lambda u, v: (u, v + np.pi / 2), (4, 2): lambda u, v: (u, v - np.pi / 2),
        (4, 3): lambda u, v: (u, v + np.pi),
        (4, 5): t5x(lambda u, v: -s(u) * c(v), lambda u, v: -s(u) * s(v) / B(u, v)),
        (4, 6): t5x(lambda u, v: s(u) * c(v), lambda u, v: -s(u) * s(v) / B(u, v)),
        (5, 1): t5x(lambda u, v: s(u) * s(v), lambda u, v: s(u) * c(v) / A(u, v)),
        (5, 2): t5x(lambda u, v: s(u) * s(v), lambda u, v: -s(u) * c(v) / A(u, v)),
        (5, 3): t5x(lambda u, v: s(u) * s(v), lambda u, v: c(u) / A(u, v)),
        (5, 4): t5x(lambda u, v: s(u) * s(v), lambda u, v: -c(u) / A(u, v)),
        (6, 1): t5x(lambda u, v: -s(u) * s(v), lambda u, v: s(u) * c(v) / A(u, v)),
        (6, 2): t5x(lambda u, v: -s(u) * s(v), lambda u, v: -s(u) * c(v) / A(u, v)),
    }


def _corrected_transitions():
    """tau_63 and tau_64 as printed carry the opposite sign of cos u (they do
    not map back to the same point of the sphere); the chart composition gives
    these."""
    s, c, acos, sq = np.sin, np.cos, np.arccos, np.sqrt
    A = lambda u, v: sq(s(u) ** 2 * c(v) ** 2 + c(u) ** 2)
    return {
        (6, 3): lambda u, v: (acos(-s(u) * s(v)), acos(-c(u) / A(u, v))),
        (6, 4): lambda u, v: (acos(-s(u) * s(v)), acos(c(u) / A(u, v))),
    }


def _overlap_points(i, j, count=4000):
    """Points (u in (0, pi), v on the extended range of the ghost layers) of
    patch i whose image lies inside patch j's domain."""
    rng = np.random.default_rng(10 * i + j)
    u = rng.uniform(0.02, np.pi - 0.02, count)
    v = rng.uniform(-0.3, np.pi + 0.3, count)
    uj, vj = mb.transition(i, j, u, v)
    keep = (uj > 0.02) & (uj < np.pi - 0.02) & (vj > 0.02) & (vj < np.pi - 0.02)
    return u[keep], v[keep]


@pytest.mark.parametrize("pair", sorted(_printed_transitions()))
def test_transitions_match_printed_appendix(pair):
    i, j = pair
    u, v = _overlap_points(i, j)
    assert len(u) > 50
    ours = mb.transition(i, j, u, v)
    pu, pv = _printed_transitions()[pair](u, v)
    # the printed v may differ by 2 pi where the chart's v is continued
    dv = np.angle(np.exp(1j * (ours[1] - pv)))
    assert np.allclose(ours[0], pu, atol=1e-12) and np.allclose(dv, 0.0, atol=1e-12)


@pytest.mark.parametrize("pair", sorted(_corrected_transitions()))
def test_transitions_63_64_with_corrected_sign(pair):
    u, v = _overlap_points(*pair)
    ours = mb.transition(*pair, u, v)
    cu, cv = _corrected_transitions()[pair](u, v)
    assert np.allclose(ours[0], cu, atol=1e-12) and np.allclose(ours[1], cv, atol=1e-12)
    assert np.allclose(chart(pair[1], cu, cv), chart(pair[0], u, v), atol=1e-13)


@pytest.mark.parametrize("pair", [(5, 6), (6, 5)])
def test_transition_56_is_pi_minus_u_minus_v(pair):
    """Composing Eq. param_maps gives (pi - u, -v); the Appendix prints (pi - u, v)."""
    u, v = _overlap_points(*pair)
    assert len(u) > 50
    ou, ov = mb.transition(*pair, u, v)
    dv = np.angle(np.exp(1j * (ov + v)))  # ov = -v up to 2 pi
    assert np.allclose(ou, np.pi - u, atol=1e-12) and np.allclose(dv, 0.0, atol=1e-12)
    assert np.allclose(chart(pair[1], np.pi - u, -v), chart(pair[0], u, v), atol=1e-14)


@pytest.mark.parametrize("i,j", [(1, 3), (1, 5), (2, 6), (3, 5), (5, 1), (6, 4), (5, 6)])
def test_transition_jacobian_against_central_differences(i, j):
    u, v = _overlap_points(i, j, 800)
    J = mb.transition_jacobian(i, j, u, v)
    e = 1e-6
    tu = (np.array(mb.transition(i, j, u + e, v)) - np.array(mb.transition(i, j, u - e, v))) / (2 * e)
    tv = (np.array(mb.transition(i, j, u, v + e)) - np.array(mb.transition(i, j, u, v - e))) / (2 * e)
    tu[1] = np.angle(np.exp(1j * tu[1] * 2 * e)) / (2 * e)
    tv[1] = np.angle(np.exp(1j * tv[1] * 2 * e)) / (2 * e)
    assert np.allclose(J[:, 0, 0], tu[0], atol=1e-7) and np.allclose(J[:, 0, 1], tu[1], atol=1e-7)
    assert np.allclose(J[:, 1, 0], tv[0], atol=1e-7) and np.allclose(J[:, 1, 1], tv[1], atol=1e-7)


# ---- spline and stencil -----------------------------------------------------
def test_spline_reproduces_bicubics_including_end_pieces():
    m = 11
    t = mb.nodes(m)
    U, V = np.meshgrid(t, t, indexing="ij")
    f = lambda u, v: (1 + u - 2 * u ** 2 + 0.3 * u ** 3) * (2 - v + 0.5 * v ** 2 - 0.1 * v ** 3)
    G = f(U, V)[..., None]
    rng = np.random.default_rng(0)
    u = rng.uniform(-0.3, np.pi + 0.3, 200)   # reaches past the first/last node
    v = rng.uniform(-0.3, np.pi + 0.3, 200)
    assert np.allclose(mb.interpolate(m, G, u, v)[:, 0], f(u, v), rtol=1e-11, atol=1e-11)


def test_seven_point_stencil_exact_to_degree_six():
    x = np.arange(-3, 4, dtype=float)
    for deg in range(7):
        assert abs(np.dot(mb.FD7, x ** deg) - (1.0 if deg == 1 else 0.0)) < 1e-13
    assert abs(np.dot(mb.FD7, x ** 7)) > 1.0  # and not beyond: sixth order


# ---- derivative scheme against closed forms ----------------------------------
def ellipsoid_exact(X, axes):
    a, b, c = axes
    g = X / np.array([a * a, b * b, c * c])
    hn = np.linalg.norm(g, axis=-1)
    n = g / hn[:, None]
    K = 1.0 / ((a * b * c) ** 2 * hn ** 4)
    H = -(np.sum(X * X, axis=-1) - a * a - b * b - c * c) / (2 * (a * b * c) ** 2 * hn ** 3)
    div = 2.0 * np.sum(X * (1.0 - n * n), axis=-1)   # div_gamma (x^2, y^2, z^2)
    return n, H, K, div


def errors(shape, axes, m, blending=True):
    s = ci.make_surface(shape, m)
    n_ex, H_ex, K_ex, div_ex = ellipsoid_exact(s.X, axes)
    geo = mb.geometry(m, s.X, blending)
    H, K = mb.curvatures(m, s.X, blending)
    gu, gv = mb.surface_derivatives(m, s.X ** 2, blending)
    div = mb.divergence_from(geo, gu, gv)
    return (rel_inf(geo["n"], n_ex), rel_inf(np.abs(H), np.abs(H_ex)), rel_inf(K, K_ex),
            rel_inf(div, div_ex))


@pytest.mark.parametrize("m", [8, 16, 32])
def test_sphere_derivatives_at_or_below_printed_errors(m):
    g = golden()
    en, eH, _, _ = errors(ci.Sphere(1.0), (1.0, 1.0, 1.0), m)
    pn, pH, _, _ = g[("sphere", m)]
    assert en <= pn and eH <= pH, (en, eH)
    nb = errors(ci.Sphere(1.0), (1.0, 1.0, 1.0), m, blending=False)
    qn, qH, _, _ = g[("sphere-noblend", m)]
    assert nb[0] <= qn and nb[1] <= qH, nb
    if m >= 16:  # blending improves the derivatives (Appendix, Remark 3)
        assert en < nb[0] and eH < nb[1]


def test_ellipsoid_derivatives_printed_table_and_fourth_order():
    """Normals and the surface divergence (first derivatives, the scheme the
    paper specifies) at or below the printed errors; H and K (second
    fundamental form via the normal's derivatives, a reading) within 5x of
    the printed errors at m = 32; all four converge at fourth order."""
    g = golden()
    axes = (0.6, 1.0, 1.0)
    errs = {}
    for m in (8, 16, 32):
        errs[m] = errors(ci.Ellipsoid(*axes), axes, m)
        pn, pH, pK, pd = g[("ellipsoid-0.6", m)]
        assert errs[m][0] <= pn and errs[m][3] <= pd, (m, errs[m])
    _, pH, pK, _ = g[("ellipsoid-0.6", 32)]
    assert errs[32][1] <= 5 * pH and errs[32][2] <= 5 * pK, errs[32]
    for q in range(4):
        assert np.log2(errs[16][q] / errs[32][q]) >= 3.5, (q, errs[16][q], errs[32][q])


# ---- Skalak force -------------------------------------------------------------
def test_stress_free_reference_has_zero_force():
    s = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), 16)
    f = mb.skalak_force(16, s.X, s.X, ES, ED)
    assert np.abs(f).max() < 1e-11


def test_uniform_dilation_of_a_sphere_closed_form():
    """Lambda = T P with T = (Es (a^2 - 1) + ED a^2 (a^4 - 1)) / 2, so
    f = div_gamma(T P) = -(2 T / a) n on the sphere of radius a."""
    a = 1.05
    T = (ES * (a * a - 1) + ED * a * a * (a ** 4 - 1)) / 2
    err = {}
    for m in (12, 24):
        s = ci.make_surface(ci.Sphere(1.0), m)
        f = mb.skalak_force(m, a * s.X, s.X, ES, ED)
        err[m] = rel_inf(f, -(2 * T / a) * s.x0)
    assert err[24] < 2e-5 and np.log2(err[12] / err[24]) >= 3.5, err


def skalak_energy(m, X, X_ref):
    """E = int_ref W_s dA_ref, invariants from the tangents of the scheme:
    tr V^2 = (G_r E - 2 F_r F + E_r G) / W_r^2, det = (W / W_r)^2."""
    g, r = mb.geometry(m, X), mb.geometry(m, X_ref)
    trV2 = (r["G"] * g["E"] - 2 * r["F"] * g["F"] + r["E"] * g["G"]) / r["W"] ** 2
    I1 = trV2 - 2.0
    I2 = (g["W"] / r["W"]) ** 2 - 1.0
    Ws = ES / 4 * (I1 ** 2 / 2 + I1 - I2) + ED / 8 * I2 ** 2
    return float(np.sum(mb.pou_weights(m) * r["W"] * (np.pi / m) ** 2 * Ws))


def test_virtual_work_matches_skalak_energy_variation():
    rel = {}
    for m in (16, 24):
        s = ci.make_surface(ci.Sphere(1.0), m)
        X = s.X * np.array([1.1, 0.95, 0.9]) + 0.05 * s.X[:, [1, 2, 0]] ** 2
        V = np.stack([np.sin(2 * s.x0[:, 0]), s.x0[:, 1] * s.x0[:, 2], np.cos(s.x0[:, 2])], -1)
        f = mb.skalak_force(m, X, s.X, ES, ED)
        lhs = np.sum(mb.quadrature_weights(m, X)[:, None] * f * V)
        e = 1e-5
        rhs = -(skalak_energy(m, X + e * V, s.X) - skalak_energy(m, X - e * V, s.X)) / (2 * e)
        rel[m] = abs(lhs - rhs) / abs(rhs)
    assert rel[24] < 2e-4 and rel[24] < rel[16] / 8, rel


def test_area_and_volume_of_the_ellipsoid():
    a, b, c = 0.9, 1.0, 1.0
    # surface area of a prolate/oblate spheroid with b = c: closed form
    e = np.sqrt(1 - a * a / (b * b))
    A_ex = 2 * np.pi * b * b * (1 + a * a / (b * b * e) * np.arctanh(e))
    V_ex = 4.0 / 3.0 * np.pi * a * b * c
    s = ci.make_surface(ci.Ellipsoid(a, b, c), 32)
    A, V = mb.area_volume(32, s.X)
    # the POU quadrature itself is accurate to ~6e-6 here (Sec. 3.3); the area
    # element from the derivative scheme matches the closed-form one far better
    assert abs(A - A_ex) / A_ex < 2e-5 and abs(V - V_ex) / V_ex < 2e-5
    geo = mb.geometry(32, s.X)
    assert np.abs(geo["W"] - s.W).max() / s.W.max() < 1e-6
