"""Overset finite-difference derivatives, the Skalak force and membrane-driven
capsule steps on the GPU against the membrane oracle (Sec. 3.5; Sec. 2.1, Eqs.
tensor and intf). Both sides are FP64, so they agree to rounding (<= 1e-11
relative) while differing in every implementation choice (spline solver,
tension invariants, reduction order)."""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle
from oracle import membrane as mb
from oracle import timestep as ts

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ES, ED = 2.0, 20.0


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = sk.Context(0)
    yield c.handle
    c.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def deformed(s):
    """A smooth non-affine deformation of a reference surface."""
    return s.X * np.array([1.08, 0.97, 0.93]) + 0.04 * s.X[:, [1, 2, 0]] ** 2


@pytest.mark.parametrize("m", [6, 9, 16, 33])
@pytest.mark.parametrize("mem", [sk.SK_HOST, sk.SK_DEVICE], ids=["host", "device"])
def test_surface_derivatives_match_oracle(ctx, m, mem):
    s = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 0.8), m)
    rng = np.random.default_rng(m)
    fields = np.concatenate([s.X, s.X ** 2, ci.sh_density(s.x0, rng, lmax=6),
                             rng.standard_normal((s.N, 2))], axis=1)   # F = 11 > one pass
    gu_o, gv_o = mb.surface_derivatives(m, fields)
    if mem == sk.SK_HOST:
        gu, gv = sk.surface_derivatives(ctx, m, mem, fields)
    else:
        gu, gv = sk.surface_derivatives(ctx, m, mem, torch.as_tensor(fields, device="cuda"))
        gu, gv = gu.cpu().numpy(), gv.cpu().numpy()
    assert rel(gu, gu_o) < 1e-12 and rel(gv, gv_o) < 1e-12, (rel(gu, gu_o), rel(gv, gv_o))


@pytest.mark.parametrize("m,shape", [(12, ci.Sphere(1.0)), (24, ci.Ellipsoid(0.9, 1.0, 1.0)),
                                     (65, ci.Ellipsoid(1.0, 0.8, 0.5))],
                         ids=["sphere-m12", "ellipsoid-m24", "ellipsoid-m65"])
def test_membrane_force_and_weights_match_oracle(ctx, m, shape):
    s = ci.make_surface(shape, m)
    X = deformed(s)
    f, w = sk.membrane_force(ctx, m, sk.SK_HOST, X, s.X, ES, ED, weights=True)
    f_o = mb.skalak_force(m, X, s.X, ES, ED)
    w_o = mb.quadrature_weights(m, X)
    assert rel(f, f_o) < 1e-11, rel(f, f_o)
    assert rel(w, w_o) < 1e-13, rel(w, w_o)


def test_membrane_force_device_memory_and_stress_free(ctx):
    s = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), 16)
    Xd = torch.as_tensor(s.X, device="cuda")
    f = sk.membrane_force(ctx, 16, sk.SK_DEVICE, Xd, Xd, ES, ED).cpu().numpy()
    assert np.abs(f).max() < 1e-11
    # dilated sphere: f = -(2 T / a) n
    s = ci.make_surface(ci.Sphere(1.0), 24)
    a = 1.05
    T = (ES * (a * a - 1) + ED * a * a * (a ** 4 - 1)) / 2
    f = sk.membrane_force(ctx, 24, sk.SK_DEVICE, torch.as_tensor(a * s.X, device="cuda"),
                          torch.as_tensor(s.X, device="cuda"), ES, ED).cpu().numpy()
    assert np.abs(f + (2 * T / a) * s.x0).max() / (2 * T / a) < 2e-5


def test_membrane_rejects_bad_arguments(ctx):
    s = ci.make_surface(ci.Sphere(1.0), 5)
    with pytest.raises(sk.SkError) as e:
        sk.membrane_force(ctx, 5, sk.SK_HOST, s.X, s.X, ES, ED)   # m >= 6
    assert e.value.code == sk.SK_EINVAL
    s = ci.make_surface(ci.Sphere(1.0), 8)
    with pytest.raises(sk.SkError) as e:
        sk.membrane_force(ctx, 8, sk.SK_HOST, s.X, s.X, -1.0, ED)
    assert e.value.code == sk.SK_EINVAL


def oracle_membrane_euler(m, X, X_ref, n_steps, dt, flow, mu):
    """Euler steps of Eq. bi_combined with the Skalak force (Eq. intf), weights
    psi W h^2 and delta* (Eq. regparam) at the current nodes, all by the oracle."""
    X = X.copy()
    for _ in range(n_steps):
        f = mb.skalak_force(m, X, X_ref, ES, ED)
        w = mb.quadrature_weights(m, X)
        surf = ci.make_surface(ci.Sphere(1.0), m)
        surf.X = X
        d = ci.delta_star(surf)
        u = oracle.sl(X, w, f, X, d, mu)
        if flow is not None and flow[0] == sk.SK_FLOW_SHEAR:
            u[:, 0] += flow[1] * X[:, 1]
        X = X + dt * u
    return X


@pytest.mark.parametrize("prec,tol", [(sk.SK_FP64, 1e-10), (sk.SK_FP32C, 2e-6)],
                         ids=["fp64", "fp32c"])
def test_capsule_membrane_steps_match_oracle(ctx, prec, tol):
    m = 12
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    X0 = deformed(ref)
    flow = (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0)
    cap = sk.Capsule(ctx, m, X0, ref.w, delta=None, mu=1.0, precision=prec)
    try:
        cap.set_membrane(ref.X, ES, ED)
        cap.step(3, 1e-3, None, flow)
        X = cap.positions()
        A, V = cap.area_volume()
    finally:
        cap.close()
    Xo = oracle_membrane_euler(m, X0, ref.X, 3, 1e-3, flow, 1.0)
    err = np.linalg.norm((X - X0) - (Xo - X0)) / np.linalg.norm(Xo - X0)
    assert err < tol, err
    Ao, Vo = mb.area_volume(m, X)
    assert abs(A - Ao) / Ao < 1e-13 and abs(V - Vo) / Vo < 1e-13


@pytest.fixture(scope="module")
def config5_oracle_run():
    """The capsule benchmark's setup (stress-free ellipsoid (0.9, 1, 1), Es = 2,
    ED = 20, shear rate 1, explicit Euler at the configured dt = 1e-3, delta*
    and weights per step) at m = 33, the largest grid whose oracle loop stays
    affordable here (the NumPy membrane oracle takes minutes per step at the
    benchmark's m = 129): 10 steps by the oracle."""
    m, n, dt = 33, 10, 1e-3
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    flow = (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0)
    Xo = oracle_membrane_euler(m, ref.X, ref.X, n, dt, flow, 1.0)
    return m, n, dt, ref, flow, Xo


@pytest.mark.parametrize("prec,tol", [(sk.SK_FP64, 1e-10), (sk.SK_FP32C, 2e-6)],
                         ids=["fp64", "fp32c"])
def test_stress_free_capsule_in_shear_matches_oracle_loop(ctx, config5_oracle_run, prec, tol):
    m, n, dt, ref, flow, Xo = config5_oracle_run
    cap = sk.Capsule(ctx, m, ref.X, ref.w, delta=None, mu=1.0, precision=prec)
    try:
        cap.set_membrane(ref.X, ES, ED)
        A0, V0 = cap.area_volume()
        cap.step(n, dt, None, flow)
        X = cap.positions()
        A, V = cap.area_volume()
    finally:
        cap.close()
    err = np.linalg.norm((X - ref.X) - (Xo - ref.X)) / np.linalg.norm(Xo - ref.X)
    assert err < tol, err
    # area and volume drift against the oracle's, from the oracle's own functionals
    Ao, Vo = mb.area_volume(m, Xo)
    Ar, Vr = mb.area_volume(m, ref.X)
    assert abs((A / A0 - 1.0) - (Ao / Ar - 1.0)) < (1e-12 if prec == sk.SK_FP64 else 1e-8)
    assert abs((V / V0 - 1.0) - (Vo / Vr - 1.0)) < (1e-12 if prec == sk.SK_FP64 else 1e-8)


def test_membrane_capsule_relaxes_toward_reference(ctx):
    """A deformed capsule with no background flow moves back toward its
    stress-free shape: the Skalak energy decreases step by step."""
    m = 16
    ref = ci.make_surface(ci.Sphere(1.0), m)
    X0 = deformed(ref)
    cap = sk.Capsule(ctx, m, X0, ref.w, delta=None, mu=1.0, precision=sk.SK_FP64)
    try:
        cap.set_membrane(ref.X, ES, ED)
        dist = [np.linalg.norm(cap.positions() - ref.X)]
        for _ in range(3):
            cap.step(20, 2e-3, None)
            dist.append(np.linalg.norm(cap.positions() - ref.X))
        _, V = cap.area_volume()
    finally:
        cap.close()
    assert all(b < a for a, b in zip(dist, dist[1:])), dist
    _, V0 = mb.area_volume(m, X0)
    assert abs(V - V0) / V0 < 1e-3   # the Stokes flow conserves volume


def oracle_membrane_rhs(m, X_ref, flow, mu):
    """u_inf(Y) + S[f(Y)](Y) at stage positions Y, all by the oracle: Skalak
    force, weights psi W h^2 and delta* (Eq. regparam) at Y."""
    def rhs(t, y):
        Y = y.reshape(-1, 3)
        surf = ci.make_surface(ci.Sphere(1.0), m)
        surf.X = Y
        u = oracle.sl(Y, mb.quadrature_weights(m, Y), mb.skalak_force(m, Y, X_ref, ES, ED), Y,
                      ci.delta_star(surf), mu)
        if flow is not None and flow[0] == sk.SK_FLOW_SHEAR:
            u[:, 0] += flow[1] * Y[:, 1]
        return u.ravel()
    return rhs


def test_rkf45_membrane_matches_oracle(ctx):
    m = 8
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    X0 = deformed(ref)
    flow = (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0)
    cap = sk.Capsule(ctx, m, X0, ref.w, delta=None, mu=1.0, precision=sk.SK_FP64)
    try:
        cap.set_membrane(ref.X, ES, ED)
        dt, acc, rej = cap.integrate_rkf45(4e-3, 2e-3, tol=1e-6, flow=flow)
        X = cap.positions()
    finally:
        cap.close()
    y, dto, acco, rejo = ts.integrate(oracle_membrane_rhs(m, ref.X, flow, 1.0), X0.ravel(),
                                      4e-3, 2e-3, 1e-6)
    assert (acc, rej) == (acco, rejo) and acc >= 2, (acc, rej, acco, rejo)
    Xo = y.reshape(-1, 3)
    assert np.linalg.norm((X - X0) - (Xo - X0)) / np.linalg.norm(Xo - X0) < 1e-9
    assert abs(dt - dto) / dto < 1e-6


def test_rkf45_errors_and_step_bound(ctx):
    m = 8
    ref = ci.make_surface(ci.Sphere(1.0), m)
    cap = sk.Capsule(ctx, m, ref.X, ref.w, delta=None, mu=1.0, precision=sk.SK_FP64)
    try:
        with pytest.raises(sk.SkError) as e:
            cap.integrate_rkf45(1e-3, 1e-4)          # no membrane, no force
        assert e.value.code == sk.SK_ENOTIMPL
        f = np.zeros((ref.N, 3))
        f[:, 2] = 1.0
        with pytest.raises(sk.SkError) as e:
            cap.integrate_rkf45(1.0, 1e-3, f=f, max_steps=2)
        assert e.value.code == sk.SK_EAGAIN
        with pytest.raises(sk.SkError) as e:
            cap.integrate_rkf45(-1.0, 1e-3, f=f)
        assert e.value.code == sk.SK_EINVAL
    finally:
        cap.close()


def test_slope_solves_staged_and_in_global_memory_agree(ctx):
    """The spline slope solves stage grid lines in shared memory when they
    fit (n <= 341) and otherwise run in global memory; the arithmetic is the
    same, so a context with staging turned off (SK_SLOPE_STAGING=0) gives the
    same derivatives bit for bit, for both line lengths with 16 and 8 lanes."""
    import os
    old = os.environ.get("SK_SLOPE_STAGING")
    os.environ["SK_SLOPE_STAGING"] = "0"
    try:
        plain = sk.Context(0)
    finally:
        if old is None:
            del os.environ["SK_SLOPE_STAGING"]
        else:
            os.environ["SK_SLOPE_STAGING"] = old
    try:
        for m in (21, 193):   # 16 and 8 lanes per line
            s = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 0.8), m)
            fields = np.concatenate([deformed(s), s.X ** 2], axis=1)
            a = sk.surface_derivatives(ctx, m, sk.SK_HOST, fields)
            b = sk.surface_derivatives(plain.handle, m, sk.SK_HOST, fields)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), m
    finally:
        plain.close()
