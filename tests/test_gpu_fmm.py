"""Single-level FMM (Sec. 5) on the GPU against the oracle's FMM (same
algorithm and decisions; independent implementations of the Tikhonov solve,
the sums and k-means) and against the direct FP64 evaluation."""

import numpy as np
import pytest

import capsule_inputs as ci
from oracle import fmm

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def seeds(s, k):
    act = np.flatnonzero(s.w)
    return s.X[act[:: max(1, len(act) // k)][:k]].copy()


@pytest.mark.parametrize("p", [4, 6])
def test_fmm_matches_oracle_fmm(ctx, p):
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 24)
    f = ci.sh_density(s.x0, np.random.default_rng(3), lmax=6)
    c0 = seeds(s, 30)
    tgt = s.X[::3]
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, tgt, 0.02, 1.2, c0, 8, p)
    ref = fmm.sl_fmm(s.X, s.w, f, tgt, 0.02, 1.2, c0, 8, p)
    assert rel(u, ref) < 1e-8, rel(u, ref)


def test_all_near_equals_direct_fp64(ctx):
    s = ci.make_surface(ci.Sphere(1.0), 12)
    f = ci.sh_density(s.x0, np.random.default_rng(4), lmax=4)
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, s.X, 10.0, 1.0, seeds(s, 8), 4, 4)
    d = sk.stokes_sl_eval(ctx, sk.SK_FP64, sk.SK_HOST, s.X, s.w, f, s.X, 10.0, 1.0)
    assert rel(u, d) < 1e-13


def test_fmm_against_direct_at_larger_size_and_device_memory(ctx):
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 65)
    f = ci.sh_density(s.x0, np.random.default_rng(5), lmax=8)
    delta = 2 * s.h
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_DEVICE, t(s.X), t(s.w), t(f), t(s.X),
                              t(np.array([delta])), 1.0, t(seeds(s, 100)), 10, 6).cpu().numpy()
    d = sk.stokes_sl_eval(ctx, sk.SK_FP64, sk.SK_HOST, s.X, s.w, f, s.X, delta, 1.0)
    assert rel(u, d) < 1e-5, rel(u, d)


def test_fmm_rejects_bad_arguments(ctx):
    s = ci.make_surface(ci.Sphere(1.0), 8)
    f = np.zeros((s.N, 3))
    for kw in ({"p": 2}, {"p": 11}):
        with pytest.raises(sk.SkError) as e:
            sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, s.X, 0.1, 1.0, seeds(s, 4), 2,
                                  **kw)
        assert e.value.code == sk.SK_EINVAL
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, s.X, -0.1, 1.0, seeds(s, 4), 2, 4)
    assert e.value.code == sk.SK_EINVAL
