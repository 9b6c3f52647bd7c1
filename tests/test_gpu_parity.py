"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (relative L2 over all targets x 3 components, the error measure of
the benchmark): SK_FP64 <= 1e-12, SK_FP32C <= 1e-6. Element-wise, every
component must also be within ATOL_FP32 * max|u| (FP32C) resp. 1e-12 * max|u|
(FP64).
"""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {sk.SK_FP64: 1e-12, sk.SK_FP32C: 1e-6}
ELEM = {sk.SK_FP64: 1e-12, sk.SK_FP32C: 1e-5}


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_close(u, ref, prec):
    assert np.all(np.isfinite(u))
    e = rel_l2(u, ref)
    assert e <= TOL[prec], f"rel-L2 {e:.3e} > {TOL[prec]:.0e}"
    scale = max(np.abs(ref).max(), 1e-300)
    emax = np.abs(u - ref).max() / scale
    assert emax <= ELEM[prec], f"max element error {emax:.3e} (of max|u|)"
    return e


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = sk.Context(0)
    yield c.handle
    c.close()


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def expected_fused(M):
    """Whether an SK_FP32C evaluation with M targets finishes its target
    blocks inside the pair kernel: at least 2 blocks (1024 targets above
    131,072 targets, else 512) per SM."""
    per_block = 1024 if M > 131072 else 512
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return -(-M // per_block) >= 2 * sms


PRECS = [sk.SK_FP64, sk.SK_FP32C]
PREC_ID = {sk.SK_FP64: "fp64", sk.SK_FP32C: "fp32c"}


@pytest.fixture(scope="module")
def sphere():
    w = ci.sphere_noise_workload()
    s = w.surface
    ref = oracle.sl(s.X, s.w, w.f, w.targets, w.delta, w.mu)
    return w, ref


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
@pytest.mark.parametrize("mem", [sk.SK_HOST, sk.SK_DEVICE], ids=["host", "device"])
def test_sl_sphere_noise(ctx, sphere, prec, mem):
    w, ref = sphere
    s = w.surface
    if mem == sk.SK_HOST:
        u = sk.stokes_sl_eval(ctx, prec, mem, s.X, s.w, w.f, w.targets, w.delta, w.mu)
    else:
        u = sk.stokes_sl_eval(ctx, prec, mem, to_dev(s.X), to_dev(s.w), to_dev(w.f),
                              to_dev(w.targets), to_dev(w.delta), w.mu).cpu().numpy()
    assert_close(u, ref, prec)
    st = sk.sk_last_eval_stats(ctx)
    assert st["n_src_active"] == s.n_active and st["n_tgt"] == s.N


@pytest.fixture(scope="module")
def rbc():
    w = ci.rbc_workload()
    s = w.surface
    ref_sl = oracle.sl(s.X, s.w, w.f, w.targets, w.delta, w.mu)
    ref_dl = oracle.dl(s.X, s.w, s.n, w.q, w.targets, w.delta)
    return w, ref_sl, ref_dl


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_sl_rbc(ctx, rbc, prec):
    w, ref, _ = rbc
    s = w.surface
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, s.X, s.w, w.f, w.targets, w.delta, w.mu)
    assert_close(u, ref, prec)
    if prec == sk.SK_FP32C:  # 48 target blocks: separate finish kernels
        assert sk.sk_last_eval_stats(ctx)["finish_fused"] == expected_fused(w.targets.shape[0])


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_dl_rbc(ctx, rbc, prec):
    w, _, ref = rbc
    s = w.surface
    u = sk.stokes_dl_eval(ctx, prec, sk.SK_HOST, s.X, s.w, s.n, w.q, w.targets, w.delta)
    assert_close(u, ref, prec)


@pytest.fixture(scope="module")
def ellipsoid_full():
    # full-size workload: 393,216 nodes + 100,000 exterior probes, delta = 2h
    return ci.ellipsoid_hires_workload()


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_sl_ellipsoid_full_size_sampled(ctx, ellipsoid_full, prec):
    w = ellipsoid_full
    s = w.surface
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_DEVICE, to_dev(s.X), to_dev(s.w), to_dev(w.f),
                          to_dev(w.targets), to_dev(w.delta), w.mu).cpu().numpy()
    if prec == sk.SK_FP32C:  # 482 target blocks: the pair kernel finishes them
        assert sk.sk_last_eval_stats(ctx)["finish_fused"] == expected_fused(w.targets.shape[0])
    rng = np.random.default_rng(77)
    M = w.targets.shape[0]
    idx = np.concatenate([rng.choice(w.n_on_surface, 384, replace=False),
                          w.n_on_surface + rng.choice(M - w.n_on_surface, 128, replace=False)])
    ref = oracle.sl(s.X, s.w, w.f, w.targets[idx], w.delta, w.mu)
    assert_close(u[idx], ref, prec)
    assert np.all(np.isfinite(u))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_sl_ellipsoid_full_size_delta_3h(ctx, ellipsoid_full, prec):
    """The headline workload at its widest regularization, delta = 3h: up to
    ~64 near pairs per target (rho < rho_T) against 96 list slots, and the
    exterior probes closest to the surface (~0.1h, nearly all of their pairs
    inside rho_c delta) among the sampled targets."""
    from scipy.spatial import cKDTree
    w = ellipsoid_full
    s = w.surface
    delta = np.array([3.0 * s.h])
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_DEVICE, to_dev(s.X), to_dev(s.w), to_dev(w.f),
                          to_dev(w.targets), to_dev(delta), w.mu).cpu().numpy()
    st = sk.sk_last_eval_stats(ctx)
    if prec == sk.SK_FP32C:
        assert st["overflow_targets"] == 0
    rng = np.random.default_rng(78)
    M, n_on = w.targets.shape[0], w.n_on_surface
    dist, _ = cKDTree(s.X).query(w.targets[n_on:])
    closest = n_on + np.argsort(dist)[:64]          # probes at ~0.1h
    idx = np.concatenate([rng.choice(n_on, 320, replace=False), closest,
                          n_on + rng.choice(M - n_on, 128, replace=False)])
    ref = oracle.sl(s.X, s.w, w.f, w.targets[idx], delta, w.mu)
    assert_close(u[idx], ref, prec)
    assert_close(u[closest], ref[320:384], prec)
    assert np.all(np.isfinite(u))


def test_dl_ellipsoid_sampled_with_probes(ctx):
    w = ci.ellipsoid_hires_workload(m=129, n_probes=20000, seed=3100)
    s = w.surface
    q = ci.sh_density(s.x0, np.random.default_rng(5), lmax=8)
    u = sk.stokes_dl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, s.X, s.w, s.n, q, w.targets, w.delta)
    idx = np.random.default_rng(6).choice(w.targets.shape[0], 512, replace=False)
    ref = oracle.dl(s.X, s.w, s.n, q, w.targets[idx], w.delta)
    assert_close(u[idx], ref, sk.SK_FP32C)


@pytest.mark.parametrize("shape,m", [(ci.Sphere(1.0), 257), (ci.Ellipsoid(1.0, 0.8, 0.5), 193)],
                         ids=["sphere-m257", "ellipsoid-m193"])
def test_dl_fp32c_large_grids(ctx, shape, m):
    """On the surface (x - y) . n cancels to O(r^2); the FP32 path differences
    coordinates in local frames, so the error stays at the single-layer level
    instead of growing like 1/delta with the grid."""
    s = ci.make_surface(shape, m)
    q = ci.sh_density(s.x0, np.random.default_rng(33), lmax=8)
    delta = 2 * s.h
    u = sk.stokes_dl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, to_dev(s.X), to_dev(s.w), to_dev(s.n),
                          to_dev(q), to_dev(s.X), to_dev(np.array([delta]))).cpu().numpy()
    # sphere m = 257: 384 blocks, fused finish; ellipsoid m = 193: 216, separate
    assert sk.sk_last_eval_stats(ctx)["finish_fused"] == expected_fused(s.N)
    idx = np.random.default_rng(6).choice(s.N, 384, replace=False)
    ref = oracle.dl(s.X, s.w, s.n, q, s.X[idx], delta)
    e = assert_close(u[idx], ref, sk.SK_FP32C)
    assert e <= 3e-7


@pytest.mark.parametrize("layer", ["sl", "dl"])
def test_fp32c_far_from_origin(ctx, layer):
    """Translating the whole problem by O(100) leaves the FP32 path's accuracy
    unchanged (coordinates enter the pair sums relative to local frames)."""
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 65)
    q = ci.sh_density(s.x0, np.random.default_rng(8), lmax=8)
    shift = np.array([100.0, -50.0, 25.0])
    X = s.X + shift
    delta = 2 * s.h
    if layer == "sl":
        u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, X, s.w, q, X, delta)
        ref = oracle.sl(X, s.w, q, X, delta)
    else:
        u = sk.stokes_dl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, X, s.w, s.n, q, X, delta)
        ref = oracle.dl(X, s.w, s.n, q, X, delta)
    e = assert_close(u, ref, sk.SK_FP32C)
    assert e <= 3e-7


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_ragged_sizes_and_per_target_delta(ctx, prec):
    """Single and double layer at ragged sizes (1 target, 1 source, partial
    tiles and target blocks) with one delta per target and random densities
    on random source subsets. On the surface (x - y).n cancels to O(r^2), and
    on a sparse subset the 32 sources of a segment span many delta: the
    double layer's FP32 path forms exact differences for pairs inside rho_c,
    so the error stays at the level of the smooth cases."""
    rng = np.random.default_rng(9)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.7, 0.6), 21)
    f = rng.standard_normal((s.N, 3))
    q = np.random.default_rng(19).standard_normal((s.N, 3))
    for n_src, n_tgt in ((1, 1), (7, 33), (257, 1), (300, 1025), (s.N, 1023), (s.N, 2049)):
        src = rng.choice(s.N, n_src, replace=False)
        Y = np.concatenate([s.X, s.X + 0.03 * s.n])[rng.choice(2 * s.N, n_tgt, replace=False)]
        delta = rng.uniform(0.5, 3.0, n_tgt) * s.h
        u = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, s.X[src], s.w[src], f[src], Y, delta, 1.3)
        ref = oracle.sl(s.X[src], s.w[src], f[src], Y, delta, 1.3)
        if np.abs(ref).max() == 0:
            assert np.all(u == 0)
        else:
            assert_close(u, ref, prec)
        # the double layer with the same per-target delta
        u = sk.stokes_dl_eval(ctx, prec, sk.SK_HOST, s.X[src], s.w[src], s.n[src], q[src], Y,
                              delta)
        ref = oracle.dl(s.X[src], s.w[src], s.n[src], q[src], Y, delta)
        if np.abs(ref).max() == 0:
            assert np.all(u == 0)
        else:
            assert_close(u, ref, prec)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_empty_and_degenerate_inputs(ctx, prec):
    Y = np.array([[0.1, 0.2, 0.3], [1.0, 0.0, 0.0]])
    # no targets: a no-op
    out = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, np.zeros((3, 3)), np.ones(3), np.ones((3, 3)),
                            np.zeros((0, 3)), 0.1)
    assert out.shape == (0, 3)
    # no sources, and only zero-weight sources: exactly zero
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)),
                          Y, 0.1)
    assert np.all(u == 0)
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, np.random.rand(50, 3), np.zeros(50),
                          np.random.rand(50, 3), Y, 0.1)
    assert np.all(u == 0)
    # a target on a node: the r = 0 limit of Sec. 3.4
    delta, mu = 0.2, 1.5
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, [[1.0, 2.0, 3.0]], [0.7], [[0.3, -1.2, 2.0]],
                          [[1.0, 2.0, 3.0]], delta, mu)
    lim = 16.0 / (3.0 * delta * np.sqrt(np.pi))
    ref = 0.7 * np.array([0.3, -1.2, 2.0]) * lim / (8 * np.pi * mu)
    assert np.allclose(u[0], ref, rtol=1e-13 if prec == sk.SK_FP64 else 1e-12)
    # double layer self term is zero
    u = sk.stokes_dl_eval(ctx, prec, sk.SK_HOST, [[1.0, 1.0, 1.0]], [1.0], [[0.0, 0.0, 1.0]],
                          [[1.0, 2.0, 3.0]], [[1.0, 1.0, 1.0]], 0.2)
    assert np.all(u == 0)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_ID.get)
def test_coincident_nodes_even_m(ctx, prec):
    s = ci.make_surface(ci.Sphere(1.0), 16)  # nodes of different patches coincide
    f = np.random.default_rng(2).standard_normal((s.N, 3))
    u = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, s.X, s.w, f, s.X, 2 * s.h)
    assert_close(u, oracle.sl(s.X, s.w, f, s.X, 2 * s.h), prec)


def test_validation_errors(ctx):
    X = np.zeros((2, 3))
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, X, np.ones(2), X, X, 0.0)
    assert e.value.code == sk.SK_EINVAL
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, X, np.ones(2), X, X, 0.1, mu=-1.0)
    assert e.value.code == sk.SK_EINVAL
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval(ctx, 7, sk.SK_HOST, X, np.ones(2), X, X, 0.1)
    assert e.value.code == sk.SK_EINVAL
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, X, np.ones(2), X, np.zeros((3, 3)),
                          [0.1, 0.2])
    assert e.value.code == sk.SK_EINVAL
    # a non-positive delta in device memory is detected on the device
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, to_dev(X), to_dev(np.ones(2)),
                          to_dev(X), to_dev(X + 1), to_dev([0.1, -0.2]))
    assert e.value.code == sk.SK_EINVAL
    # the context is still usable afterwards
    u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, X + [[0, 0, 1], [0, 0, 0]], np.ones(2),
                          X + 1, X + 3, 0.1)
    assert np.all(np.isfinite(u))


def test_near_list_overflow_rescan(ctx):
    """rho_T = 2 at delta = 3h puts ~300 pairs per target below rho_T: every
    list overflows and the exact FP32-classified rescan takes over."""
    s = ci.make_surface(ci.Sphere(1.0), 33)
    f = np.random.default_rng(4).standard_normal((s.N, 3))
    try:
        sk.sk_set_fp32c_thresholds(ctx, 2.0, 5.0)
        u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, s.X, s.w, f, s.X, 3 * s.h)
        st = sk.sk_last_eval_stats(ctx)
    finally:
        sk.sk_set_fp32c_thresholds(ctx, 0.5, 5.0)
    assert st["overflow_targets"] > 0
    assert_close(u, oracle.sl(s.X, s.w, f, s.X, 3 * s.h), sk.SK_FP32C)


def test_near_list_overflow_in_the_fused_finish(ctx):
    """320,000 targets near a sphere m = 33 (3960 active nodes) with rho_T = 2
    and delta = 0.28: ~300 near pairs per target, every group list overflows,
    and the pair kernel's own finish (two pairs per lane, fused) rescans."""
    s = ci.make_surface(ci.Sphere(1.0), 33)
    rng = np.random.default_rng(9)
    f = rng.standard_normal((s.N, 3))
    d = rng.standard_normal((320_000, 3))
    Y = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0.98, 1.02, (320_000, 1))
    try:
        sk.sk_set_fp32c_thresholds(ctx, 2.0, 5.0)
        u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, s.X, s.w, f, Y, 0.28)
        st = sk.sk_last_eval_stats(ctx)
    finally:
        sk.sk_set_fp32c_thresholds(ctx, 0.5, 5.0)
    assert st["finish_fused"] == 1 and expected_fused(len(Y))
    assert st["overflow_targets"] > 0
    pick = np.random.default_rng(10).choice(len(Y), 256, replace=False)
    assert_close(u[pick], oracle.sl(s.X, s.w, f, Y[pick], 0.28), sk.SK_FP32C)


def _long_list_case(n_far, seed):
    """Sphere m = 33 (3960 active nodes) with rho_T = 2: one target near all
    of them, a list longer than a warp's near-sum scratch, so the finish
    rescans it; one with ~300 near pairs (more than the 96 slots per target
    of the pooled group lists, within the group's capacity; the heapsort
    path); one with a few dozen; and n_far targets 10 away with none."""
    s = ci.make_surface(ci.Sphere(1.0), 33)
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((s.N, 3))
    near = s.X[rng.choice(s.N, 3, replace=False)] * np.array([[1.0], [1.0], [1.01]])
    far = rng.standard_normal((n_far, 3))
    far = 10.0 * far / np.linalg.norm(far, axis=1, keepdims=True) * rng.uniform(1.0, 1.5, (n_far, 1))
    Y = np.concatenate([near, far])
    delta = np.concatenate([[1.0, 0.25, s.h], np.full(n_far, s.h)])
    return s, f, Y, delta


@pytest.mark.parametrize("n_far", [61, 320_000])
def test_long_near_lists_without_overflow(ctx, n_far):
    """Near lists are pooled per target group: a target may hold far more
    than 96 near pairs as long as its group's list has room, and a target
    with more than a warp's scratch is rescanned in the finish. 64 targets
    run one pair per lane and the separate finish; 320,003 run two pairs per
    lane and the finish inside the pair kernel."""
    s, f, Y, delta = _long_list_case(n_far, 7)
    try:
        sk.sk_set_fp32c_thresholds(ctx, 2.0, 5.0)
        u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, s.X, s.w, f, Y, delta)
        st = sk.sk_last_eval_stats(ctx)
    finally:
        sk.sk_set_fp32c_thresholds(ctx, 0.5, 5.0)
    assert st["overflow_targets"] == 0
    assert st["finish_fused"] == int(expected_fused(len(Y)))
    pick = np.concatenate([[0, 1, 2], 3 + np.random.default_rng(8).choice(n_far, 61, replace=False)])
    ref = oracle.sl(s.X, s.w, f, Y[pick], delta[pick])
    assert_close(u[pick], ref, sk.SK_FP32C)
    # the three near targets against their own sums (the far ones are small)
    for i in range(3):
        assert rel_l2(u[i], ref[i]) <= 1e-6
    rho = np.linalg.norm(Y[:3, None, :] - s.X[None, s.w != 0], axis=-1) / delta[:3, None]
    n_near = (rho < 2.0).sum(axis=1)
    assert n_near[0] > 3000 and 96 < n_near[1] < 1900 and 0 < n_near[2] < 96
    assert abs(st["near_pairs"] - int(n_near.sum())) <= 3  # FP32 vs FP64 at rho = 2


@pytest.mark.parametrize("rho_T,rho_c", [(0.25, 5.0), (1.0, 5.0), (0.5, 4.5), (0.5, 6.0)])
def test_fp32c_threshold_variants(ctx, rbc, rho_T, rho_c):
    w, ref, _ = rbc
    s = w.surface
    try:
        sk.sk_set_fp32c_thresholds(ctx, rho_T, rho_c)
        u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, s.X, s.w, w.f, w.targets, w.delta)
    finally:
        sk.sk_set_fp32c_thresholds(ctx, 0.5, 5.0)
    assert_close(u, ref, sk.SK_FP32C)


def test_deterministic_and_independent_of_target_order(ctx, rbc):
    w, _, _ = rbc
    s = w.surface
    args = (s.X, s.w, w.f)
    u1 = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *args, w.targets, w.delta)
    u2 = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *args, w.targets, w.delta)
    assert np.array_equal(u1, u2)
    perm = np.random.default_rng(1).permutation(w.targets.shape[0])
    u3 = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *args, w.targets[perm], w.delta)
    assert np.array_equal(u3, u1[perm])
    # a subset of the targets gives bit-identical values
    sub = perm[:1000]
    u4 = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *args, w.targets[sub], w.delta)
    assert np.array_equal(u4, u1[sub])


def test_async_stream_device_memory(ctx, rbc):
    w, ref, _ = rbc
    s = w.surface
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        X, W, F, Y, D = (to_dev(a) for a in (s.X, s.w, w.f, w.targets, w.delta))
        out = torch.empty((Y.shape[0], 3), dtype=torch.float64, device="cuda")
    sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, X, W, F, Y, D, 1.0, u_out=out, stream=st)
    st.synchronize()
    assert_close(out.cpu().numpy(), ref, sk.SK_FP32C)


def test_stats_near_pairs_match_independent_count(ctx, rbc):
    from scipy.spatial import cKDTree
    w, _, _ = rbc
    s = w.surface
    sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, s.X, s.w, w.f, w.targets, w.delta)
    st = sk.sk_last_eval_stats(ctx)
    act = s.w != 0
    n = cKDTree(s.X[act]).query_ball_point(w.targets, r=0.5 * w.delta[0], return_length=True)
    assert abs(st["near_pairs"] - n.sum()) <= 1e-3 * n.sum()
    assert st["overflow_targets"] == 0


@pytest.mark.parametrize("layer", ["sl", "dl"])
def test_target_pairs_per_lane_boundary(ctx, layer):
    """M = 131,072 runs one f32x2 target pair per lane (3 CTAs/SM), M = 131,073
    two (2 CTAs/SM). Both match the oracle on sampled targets, and the shared
    targets agree across the two tilings up to the FP64 merge of chunk
    partials (the chunk counts differ)."""
    rng = np.random.default_rng(61)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), 65)
    dens = ci.sh_density(s.x0, rng, lmax=6)
    probes, _ = ci.exterior_probes(ci.Ellipsoid(1.0, 0.8, 0.5), 131073 - s.N, s.h, rng)
    Y = np.concatenate([s.X, probes])
    delta = np.array([2.0 * s.h])
    idx = rng.choice(131072, 384, replace=False)
    if layer == "sl":
        ref = oracle.sl(s.X, s.w, dens, Y[idx], delta, 1.0)
    else:
        ref = oracle.dl(s.X, s.w, s.n, dens, Y[idx], delta)
    outs = []
    for M in (131072, 131073):
        if layer == "sl":
            u = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, to_dev(s.X), to_dev(s.w),
                                  to_dev(dens), to_dev(Y[:M]), to_dev(delta), 1.0)
        else:
            u = sk.stokes_dl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, to_dev(s.X), to_dev(s.w),
                                  to_dev(s.n), to_dev(dens), to_dev(Y[:M]), to_dev(delta))
        u = u.cpu().numpy()
        assert_close(u[idx], ref, sk.SK_FP32C)
        outs.append(u)
    assert rel_l2(outs[1][:131072], outs[0]) < 1e-12


def test_single_block_sort_matches_multi_block_sort(ctx):
    """Small point sets are ordered by one single-block kernel, larger ones by
    fifteen launches; both run the same per-tile code, so the sorted order,
    and hence every result, is the same bit for bit. A second context with the
    single-block path turned off (SK_SMALL_SORT_POINTS=0) gives the reference;
    sizes cover 1, ragged tiles, both sides of the point limit and zero-weight
    sources."""
    import os
    old = os.environ.get("SK_SMALL_SORT_POINTS")
    os.environ["SK_SMALL_SORT_POINTS"] = "0"
    try:
        multi = sk.Context(0)
    finally:
        if old is None:
            del os.environ["SK_SMALL_SORT_POINTS"]
        else:
            os.environ["SK_SMALL_SORT_POINTS"] = old
    rng = np.random.default_rng(67)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.6), 38)   # N = 8214
    f = rng.standard_normal((s.N, 3))
    try:
        for n_src, n_tgt in ((1, 1), (33, 2047), (2048, 2049), (3072, 3073), (4095, 6000),
                             (8192, 8192),
                             (s.N, 3000)):
            src = rng.choice(s.N, n_src, replace=False)
            w = s.w[src].copy()
            w[rng.random(n_src) < 0.2] = 0.0
            Y = s.X[rng.choice(s.N, n_tgt, replace=False)] + 0.01 * rng.standard_normal((n_tgt, 3))
            for prec in PRECS:
                a = sk.stokes_sl_eval(ctx, prec, sk.SK_HOST, s.X[src], w, f[src], Y, 2 * s.h)
                b = sk.stokes_sl_eval(multi.handle, prec, sk.SK_HOST, s.X[src], w, f[src], Y,
                                      2 * s.h)
                assert np.array_equal(a, b), (n_src, n_tgt, prec)
                c = sk.stokes_dl_eval(ctx, prec, sk.SK_HOST, s.X[src], w, s.n[src], f[src], Y,
                                      2 * s.h)
                d = sk.stokes_dl_eval(multi.handle, prec, sk.SK_HOST, s.X[src], w, s.n[src],
                                      f[src], Y, 2 * s.h)
                assert np.array_equal(c, d), (n_src, n_tgt, prec)
        st = sk.sk_last_eval_stats(multi.handle)
        assert st["kernel_launches"] > 0
    finally:
        multi.close()
