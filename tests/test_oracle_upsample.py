"""Pins of the upsampled single layer (oracle/upsample.py, Sec. 3.4):

* I_u reproduces bicubic fields in (u, v) at every fine node, and returns the
  coarse values at the fine nodes that coincide with coarse ones;
* the fine POU weights integrate the sphere's area like the coarse ones;
* a sphere under uniform traction translates rigidly, S[f0] = 2 f0 / (3 mu):
  upsampling reduces the error;
* the ellipsoid (0.6, 1, 1) with f = (x^2, y^2, z^2) (Table ellipsoid_sing):
  against a finer upsampled solution at shared nodes, the errors with and
  without upsampling are at or below the printed ones, and upsampling gains
  at least the printed factor's order of magnitude.
"""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle
from conftest import read_golden
from oracle import membrane as mb
from oracle import upsample as up


def test_upsampling_is_exact_on_bicubics_and_interpolates():
    m = 9
    s = ci.make_surface(ci.Sphere(1.0), m)
    h = np.pi / m
    u, v = s.j * h, s.k * h
    f = lambda u, v: (1 + u - 0.4 * u ** 3) * (2 - v + 0.2 * v ** 2 - 0.05 * v ** 3)
    G = np.stack([f(u, v), u * v], axis=1)
    fine = up.upsample(m, G)
    mu_, fu, fv = up.fine_grid(m)
    fu = np.tile(fu, 6)
    fv = np.tile(fv, 6)
    assert np.allclose(fine[:, 0], f(fu, fv), rtol=1e-12, atol=1e-12)
    assert np.allclose(fine[:, 1], fu * fv, rtol=1e-12, atol=1e-12)
    # coarse node (j, k) is fine node (4j, 4k)
    n, nf = m - 1, mu_ - 1
    Gr = G.reshape(6, n, n, 2)
    Fr = fine.reshape(6, nf, nf, 2)
    assert np.array_equal(Fr[:, 3::4, 3::4][:, :n, :n], Gr) or \
        np.allclose(Fr[:, 3::4, 3::4][:, :n, :n], Gr, rtol=0, atol=1e-14)


def test_fine_weights_integrate_the_area():
    m = 12
    s = ci.make_surface(ci.Sphere(1.0), m)
    geo = mb.geometry(m, s.X)
    Wu = up.upsample(m, geo["W"])
    hu = np.pi / (4 * m)
    A = np.sum(up.fine_pou(m) * Wu * hu * hu)
    A_coarse = np.sum(s.w)
    # interpolating W costs O(h^4); the fine grid still beats the coarse sum
    assert abs(A - 4 * np.pi) / (4 * np.pi) < 3e-5
    assert abs(A - 4 * np.pi) < abs(A_coarse - 4 * np.pi) / 10


def test_uniform_traction_on_a_sphere_improves_with_upsampling():
    m = 10
    s = ci.make_surface(ci.Sphere(1.0), m)
    f = np.zeros((s.N, 3))
    f[:, 2] = 1.0
    exact = 2.0 / 3.0
    u_up = up.sl_upsampled(m, s.X, s.W, f)
    e_up = np.abs(u_up[:, 2] - exact).max() / exact
    u = oracle.sl(s.X, s.w, f, s.X, ci.delta_star(s))
    e = np.abs(u[:, 2] - exact).max() / exact
    assert e_up < e / 5 and e_up < 2e-3, (e, e_up)


@pytest.fixture(scope="module")
def ellipsoid_reference():
    """S[(x^2, y^2, z^2)] on the ellipsoid (0.6, 1, 1) at the m = 8 nodes from
    the upsampled sum on the m = 48 grid (the m = 8 nodes are m = 48 nodes)."""
    axes = (0.6, 1.0, 1.0)
    m_ref = 48
    s = ci.make_surface(ci.Ellipsoid(*axes), m_ref)
    W = mb.geometry(m_ref, s.X)["W"]
    idx = _nodes_of(16, m_ref)
    u = np.full((s.N, 3), np.nan)
    u[idx] = up.sl_upsampled(m_ref, s.X, W, s.X ** 2, targets=idx)
    n = m_ref - 1
    return axes, u.reshape(6, n, n, 3)


def _nodes_of(m, m_ref=48):
    """Indices, in the m_ref grid, of the nodes of the m-th order grid."""
    step = m_ref // m
    n, nr = m - 1, m_ref - 1
    p, j, k = np.meshgrid(np.arange(6), np.arange(1, m) * step - 1, np.arange(1, m) * step - 1,
                          indexing="ij")
    return ((p * nr + j) * nr + k).ravel()


def _at_nodes_of(m, ur, m_ref=48):
    return ur.reshape(-1, 3)[_nodes_of(m, m_ref)]


@pytest.mark.parametrize("m", [8, 16])
def test_ellipsoid_single_layer_table(ellipsoid_reference, m):
    axes, ur = ellipsoid_reference
    printed = {int(r[0]): (float(r[1]), float(r[2])) for r in read_golden("single_layer_errors.txt")}
    ref = _at_nodes_of(m, ur)
    s = ci.make_surface(ci.Ellipsoid(*axes), m)
    f = s.X ** 2
    W = mb.geometry(m, s.X)["W"]  # area element by the derivative scheme, as in the paper
    e_up = np.abs(up.sl_upsampled(m, s.X, W, f) - ref).max() / np.abs(ref).max()
    w = mb.quadrature_weights(m, s.X)
    e = np.abs(oracle.sl(s.X, w, f, s.X, ci.delta_star(s)) - ref).max() / np.abs(ref).max()
    p_noup, p_up = printed[m]
    # one significant digit printed; details the paper leaves open (delta*
    # neighbourhoods, spline end conditions) move the coarsest grid by ~10%
    assert e <= 1.25 * p_noup and e_up <= p_up, (m, e, e_up)
    assert e_up < e / 5, (e, e_up)


def test_coarse_nodes_match_a_finer_upsampled_solution():
    """S[(x^2, y^2, z^2)] on the ellipsoid (0.6, 1, 1): the m = 8 upsampled sum
    against the m = 24 upsampled sum at the shared nodes stays within the error
    Table ellipsoid_sing prints for m = 8 with upsampling (its reference is the
    paper's finest grid; this one is cheaper, so the bound is the printed one)."""
    axes, m, m_ref = (0.6, 1.0, 1.0), 8, 24
    printed = {int(r[0]): float(r[2]) for r in read_golden("single_layer_errors.txt")}
    sr = ci.make_surface(ci.Ellipsoid(*axes), m_ref)
    idx = _nodes_of(m, m_ref)
    ref = up.sl_upsampled(m_ref, sr.X, mb.geometry(m_ref, sr.X)["W"], sr.X ** 2, targets=idx)
    s = ci.make_surface(ci.Ellipsoid(*axes), m)
    u = up.sl_upsampled(m, s.X, mb.geometry(m, s.X)["W"], s.X ** 2)
    e = np.abs(u - ref).max() / np.abs(ref).max()
    assert e <= printed[m], e
