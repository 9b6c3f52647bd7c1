"""capsule_step: explicit Euler steps of dx/dt = u_inf + S[f] (Eq. bi_combined).

Compared with the same Euler loop driven by the FP64 oracle: the oracle's
single layer at the current nodes, delta* of Eq. regparam from the input
generator, and the background flows of Eqs. shear_flow / poiseuille_flow.
"""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = sk.Context(0)
    yield c.handle
    c.close()


def delta_star_of(X, m):
    surf = ci.make_surface(ci.Sphere(1.0), m)
    surf.X = X
    return ci.delta_star(surf)


def u_inf(X, flow):
    u = np.zeros_like(X)
    if flow is None:
        return u
    kind, rate, alpha, R0 = flow
    if kind == sk.SK_FLOW_SHEAR:
        u[:, 0] = rate * X[:, 1]
    elif kind == sk.SK_FLOW_POISEUILLE:
        u[:, 0] = alpha * (R0 ** 2 - X[:, 1] ** 2 - X[:, 2] ** 2)
    return u


def oracle_euler(X, w, f, m, n_steps, dt, flow, mu, delta=None):
    X = X.copy()
    for _ in range(n_steps):
        d = delta_star_of(X, m) if delta is None else delta
        X = X + dt * (oracle.sl(X, w, f, X, d, mu) + u_inf(X, flow))
    return X


@pytest.mark.parametrize("prec,tol", [(sk.SK_FP64, 1e-11), (sk.SK_FP32C, 1e-6)],
                         ids=["fp64", "fp32c"])
@pytest.mark.parametrize("flow", [None, (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0),
                                  (sk.SK_FLOW_POISEUILLE, 0.0, 1.0, 5.0)],
                         ids=["none", "shear", "poiseuille"])
def test_euler_steps_match_oracle(ctx, prec, tol, flow):
    m = 13
    surf = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    f = ci.sh_density(surf.x0, np.random.default_rng(3), lmax=8)
    cap = sk.Capsule(ctx, m, surf.X, surf.w, delta=None, mu=1.3, precision=prec)
    try:
        cap.step(4, 0.01, f, flow)
        X = cap.positions()
    finally:
        cap.close()
    ref = oracle_euler(surf.X, surf.w, f, m, 4, 0.01, flow, 1.3)
    disp_ref = ref - surf.X
    err = np.linalg.norm((X - surf.X) - disp_ref) / np.linalg.norm(disp_ref)
    assert err <= tol, err


def test_fixed_delta_repeated_calls_and_errors(ctx):
    m = 9
    surf = ci.make_surface(ci.Sphere(1.0), m)
    f = np.zeros((surf.N, 3))
    f[:, 2] = 1.0  # uniform traction: the sphere translates rigidly, u = 2 f / (3 mu)
    cap = sk.Capsule(ctx, m, surf.X, surf.w, delta=[2 * surf.h], mu=1.0, precision=sk.SK_FP64)
    try:
        cap.step(3, 0.1, f)
        cap.step(2, 0.1, f)  # the captured step is reused
        X = cap.positions()
        ref = oracle_euler(surf.X, surf.w, f, m, 5, 0.1, None, 1.0, delta=2 * surf.h)
        assert np.allclose(X, ref, rtol=0, atol=1e-13)
        # rigid translation up to the quadrature error of this coarse grid
        shift = (X - surf.X).mean(axis=0)
        assert abs(shift[2] - 0.5 * 2.0 / 3.0) < 2e-2
        with pytest.raises(sk.SkError) as e:
            cap.step(1, 0.1, None)  # the Skalak force is not built
        assert e.value.code == sk.SK_ENOTIMPL
        with pytest.raises(sk.SkError) as e:
            cap.step(1, -1.0, f)
        assert e.value.code == sk.SK_EINVAL
    finally:
        cap.close()
