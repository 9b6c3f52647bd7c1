"""Single-level FMM (Sec. 5) on the GPU against the oracle's FMM (the same
algorithm and box-against-box decisions; independent implementations of the
Tikhonov solve, the sums and k-means) and against the oracle's direct sum."""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle
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


# against the oracle's FMM: FP64 to the rounding of the Tikhonov solve, FP32C
# at the FP32C tolerance of the direct sums
TOL = {sk.SK_FP64: 1e-8, sk.SK_FP32C: 1e-6}
PRECS = [sk.SK_FP64, sk.SK_FP32C]
PREC_ID = {sk.SK_FP64: "fp64", sk.SK_FP32C: "fp32c"}


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
@pytest.mark.parametrize("p", [4, 6, 8])
def test_fmm_matches_oracle_fmm(ctx, p, prec):
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 24)
    f = ci.sh_density(s.x0, np.random.default_rng(3), lmax=6)
    c0 = seeds(s, 30)
    tgt = s.X[::3]
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, tgt, 0.02, 1.2, c0, 8, p,
                              precision=prec)
    ref = fmm.sl_fmm(s.X, s.w, f, tgt, 0.02, 1.2, c0, 8, p)
    assert rel(u, ref) < TOL[prec], rel(u, ref)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_fmm_with_probes_and_per_target_delta_matches_oracle_fmm(ctx, prec):
    """Off-surface probes join the boxes of their nearest centres; per-target
    delta makes the box's largest delta decide its neighbours."""
    rng = np.random.default_rng(8)
    shape = ci.Ellipsoid(1.0, 0.8, 0.5)
    s = ci.make_surface(shape, 24)
    f = ci.sh_density(s.x0, rng, lmax=6)
    probes, _ = ci.exterior_probes(shape, 400, s.h, rng)
    tgt = np.concatenate([s.X[::4], probes])
    delta = rng.uniform(0.01, 0.03, len(tgt))
    c0 = seeds(s, 30)
    pl = fmm.plan(s.X, s.w, tgt, delta, c0, 8)
    assert 0.2 < pl["near"].mean() < 0.9     # both kinds of box pairs occur
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, tgt, delta, 0.9, c0, 8, 6,
                              precision=prec)
    ref = fmm.sl_fmm(s.X, s.w, f, tgt, delta, 0.9, c0, 8, 6)
    assert rel(u, ref) < TOL[prec], rel(u, ref)


@pytest.mark.parametrize("prec,tol", [(sk.SK_FP64, 1e-13), (sk.SK_FP32C, 1e-6)],
                         ids=["fp64", "fp32c"])
def test_all_near_equals_the_direct_sum(ctx, prec, tol):
    s = ci.make_surface(ci.Sphere(1.0), 12)
    f = ci.sh_density(s.x0, np.random.default_rng(4), lmax=4)
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, s.X, 10.0, 1.0, seeds(s, 8), 4, 4,
                              precision=prec)
    assert rel(u, fmm.sl_fmm(s.X, s.w, f, s.X, 10.0, 1.0, seeds(s, 8), 4, 4)) < tol
    assert rel(u, oracle.sl(s.X, s.w, f, s.X, 10.0, 1.0)) < tol


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_fmm_at_larger_size_and_device_memory(ctx, prec):
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 65)
    f = ci.sh_density(s.x0, np.random.default_rng(5), lmax=8)
    delta = 2 * s.h
    c0 = seeds(s, 100)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    u = sk.stokes_sl_eval_fmm(ctx, sk.SK_DEVICE, t(s.X), t(s.w), t(f), t(s.X),
                              t(np.array([delta])), 1.0, t(c0), 10, 6,
                              precision=prec).cpu().numpy()
    ref = fmm.sl_fmm(s.X, s.w, f, s.X, delta, 1.0, c0, 10, 6)
    assert rel(u, ref) < TOL[prec], rel(u, ref)
    d = oracle.sl(s.X, s.w, f, s.X, delta, 1.0)
    assert rel(u, d) < 1e-5, rel(u, d)


def test_fp32c_fmm_two_target_pairs_per_lane(ctx):
    """More than 131,072 targets (ellipsoid m = 129 nodes and 40,000 exterior
    probes): the FP32C FMM runs two target pairs per lane and groups of 128
    targets. Against the FP64 FMM (same plan: FP32 rounding only) and the
    direct oracle on sampled targets."""
    shape = ci.Ellipsoid(1.0, 0.8, 0.5)
    s = ci.make_surface(shape, 129)
    rng = np.random.default_rng(21)
    f = ci.sh_density(s.x0, rng, lmax=8)
    probes, _ = ci.exterior_probes(shape, 40_000, s.h, rng)
    Y = np.concatenate([s.X, probes])
    assert Y.shape[0] > 131_072
    delta = 2 * s.h
    c0 = seeds(s, 64)
    u32 = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, Y, delta, 1.0, c0, 10, 6,
                                precision=sk.SK_FP32C)
    u64 = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, s.w, f, Y, delta, 1.0, c0, 10, 6,
                                precision=sk.SK_FP64)
    assert rel(u32, u64) < 1e-6, rel(u32, u64)
    pick = np.random.default_rng(22).choice(Y.shape[0], 256, replace=False)
    d = oracle.sl(s.X, s.w, f, Y[pick], delta, 1.0)
    assert rel(u32[pick], d) < 1e-5, rel(u32[pick], d)


def test_fp32c_fmm_ragged_and_degenerate(ctx):
    """One cluster (all near), clusters left empty by k-means, zero weights,
    a single target, and more targets than one block; the FP32C FMM against
    the oracle's FMM."""
    rng = np.random.default_rng(12)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.9, 0.7), 17)
    f = rng.standard_normal((s.N, 3))
    w = s.w.copy()
    w[rng.random(s.N) < 0.3] = 0.0
    cases = [(s.X[:1], 1, 0.05), (s.X, 1, 0.05), (s.X[::2], 40, 0.03),
             (np.concatenate([s.X, s.X + 0.02 * s.n]), 25, 0.04)]
    for tgt, k, delta in cases:
        c0 = s.X[np.flatnonzero(w)[:: max(1, np.count_nonzero(w) // k)][:k]].copy()
        c0[-1] += 5.0          # a centre far away: its cluster may stay empty
        u = sk.stokes_sl_eval_fmm(ctx, sk.SK_HOST, s.X, w, f, tgt, delta, 1.1, c0, 6, 5,
                                  precision=sk.SK_FP32C)
        ref = fmm.sl_fmm(s.X, w, f, tgt, delta, 1.1, c0, 6, 5)
        assert rel(u, ref) < 1e-6, (len(tgt), k, rel(u, ref))


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
