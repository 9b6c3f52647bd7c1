"""Four-times upsampled single layer (Sec. 3.4) on the GPU against the oracle's
upsampled sum (oracle/upsample.py): same interpolant definition, independent
implementations (spline solver, Hermite evaluation, delta_u, the sum)."""

import numpy as np
import pytest

import capsule_inputs as ci
from oracle import membrane as mb
from oracle import upsample as up

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {sk.SK_FP64: 1e-12, sk.SK_FP32C: 1e-6}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = sk.Context(0)
    yield c.handle
    c.close()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [sk.SK_FP64, sk.SK_FP32C], ids=["fp64", "fp32c"])
@pytest.mark.parametrize("m", [8, 16, 33])
def test_upsampled_single_layer_matches_oracle(ctx, prec, m):
    s = ci.make_surface(ci.Ellipsoid(0.6, 1.0, 1.0), m)
    W = mb.geometry(m, s.X)["W"]
    f = s.X ** 2
    u = sk.stokes_sl_eval_upsampled(ctx, prec, sk.SK_HOST, m, s.X, W, f, 1.3)
    ref = up.sl_upsampled(m, s.X, W, f, 1.3)
    assert rel(u, ref) < TOL[prec], rel(u, ref)


def test_upsampled_device_memory_and_stream(ctx):
    m = 12
    s = ci.make_surface(ci.EvansFungRBC(ci.random_rotation(np.random.default_rng(2))), m)
    W = mb.geometry(m, s.X)["W"]
    f = ci.sh_density(s.x0, np.random.default_rng(3), lmax=6)
    st = torch.cuda.Stream()
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    with torch.cuda.stream(st):
        u = sk.stokes_sl_eval_upsampled(ctx, sk.SK_FP64, sk.SK_DEVICE, m, d(s.X), d(W), d(f),
                                        1.0, stream=st)
    st.synchronize()
    ref = up.sl_upsampled(m, s.X, W, f)
    assert rel(u.cpu().numpy(), ref) < 1e-12


def test_upsampling_reduces_the_sphere_translation_error(ctx):
    m = 10
    s = ci.make_surface(ci.Sphere(1.0), m)
    f = np.zeros((s.N, 3))
    f[:, 2] = 1.0
    u_up = sk.stokes_sl_eval_upsampled(ctx, sk.SK_FP64, sk.SK_HOST, m, s.X, s.W, f, 1.0)
    u = sk.stokes_sl_eval(ctx, sk.SK_FP64, sk.SK_HOST, s.X, s.w, f, s.X, ci.delta_star(s), 1.0)
    e_up = np.abs(u_up[:, 2] - 2 / 3).max()
    e = np.abs(u[:, 2] - 2 / 3).max()
    assert e_up < e / 5


def oracle_upsampled_velocity(m, X, X_ref, flow, mu, ES=2.0, ED=20.0):
    """u_inf(X) + S[f](X) with f the Skalak force and the upsampled sum."""
    W = mb.geometry(m, X)["W"]
    f = mb.skalak_force(m, X, X_ref, ES, ED)
    u = up.sl_upsampled(m, X, W, f, mu)
    if flow is not None:
        u[:, 0] += flow[1] * X[:, 1]
    return u


def test_capsule_upsampled_euler_and_rkf45_match_oracle(ctx):
    from oracle import timestep as ts
    m = 8
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    X0 = ref.X * np.array([1.05, 0.98, 0.97])
    flow = (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0)
    cap = sk.Capsule(ctx, m, X0, ref.w, delta=None, mu=1.0, precision=sk.SK_FP64)
    try:
        cap.set_membrane(ref.X, 2.0, 20.0)
        cap.set_upsampling(4)
        cap.step(2, 1e-3, None, flow)
        Xe = cap.positions()
    finally:
        cap.close()
    Xo = X0.copy()
    for _ in range(2):
        Xo = Xo + 1e-3 * oracle_upsampled_velocity(m, Xo, ref.X, flow, 1.0)
    assert rel(Xe - X0, Xo - X0) < 1e-10
    cap = sk.Capsule(ctx, m, X0, ref.w, delta=None, mu=1.0, precision=sk.SK_FP64)
    try:
        cap.set_membrane(ref.X, 2.0, 20.0)
        cap.set_upsampling(4)
        dt, acc, rej = cap.integrate_rkf45(3e-3, 1.5e-3, tol=1e-6, flow=flow)
        Xr = cap.positions()
    finally:
        cap.close()
    rhs = lambda t, y: oracle_upsampled_velocity(m, y.reshape(-1, 3), ref.X, flow, 1.0).ravel()
    y, dto, acco, rejo = ts.integrate(rhs, X0.ravel(), 3e-3, 1.5e-3, 1e-6)
    assert (acc, rej) == (acco, rejo)
    assert rel(Xr - X0, y.reshape(-1, 3) - X0) < 1e-9


def test_shape_moments_of_an_ellipsoid(ctx):
    """A, V and the inertia tensor of the ellipsoid (a, b, c) against closed
    forms: V = 4 pi abc / 3, J = V/5 diag(b^2 + c^2, a^2 + c^2, a^2 + b^2)."""
    a, b, c = 0.9, 1.0, 0.8
    m = 33
    s = ci.make_surface(ci.Ellipsoid(a, b, c), m)
    shift = np.array([12.0, -0.2, 0.1])   # far from the origin, like a capsule carried downstream
    cap = sk.Capsule(ctx, m, s.X + shift, s.w, delta=None, mu=1.0, precision=sk.SK_FP64)
    try:
        A, V, cen, J = cap.shape_moments()
    finally:
        cap.close()
    V_ex = 4 * np.pi * a * b * c / 3
    J_ex = V_ex / 5 * np.diag([b * b + c * c, a * a + c * c, a * a + b * b])
    assert abs(V - V_ex) / V_ex < 1e-5
    assert np.allclose(cen, shift, atol=1e-6)
    assert np.linalg.norm(J - J_ex) / np.linalg.norm(J_ex) < 1e-5
    Ao, Vo = mb.area_volume(m, s.X)
    assert abs(A - Ao) / Ao < 1e-12
