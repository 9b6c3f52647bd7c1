"""Continuous-batching serving through the C ABI (needs a GB300).

Each served request must equal stokes_sl_eval(SK_FP32C) on the same inputs
bit for bit (same decomposition and order of every sum), alone and in any
mix, and match the oracle within the FP32C tolerance.
"""

import time

import numpy as np
import pytest

import capsule_inputs as ci
from capsule_inputs.workloads import build_request
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


def mixed_requests(n, m_choices=(9, 13, 17, 25, 33, 49, 65), seed=41):
    rng = np.random.default_rng(seed)
    specs = ci.serving_mix(n, seed=seed)
    out = []
    for s in specs:
        s["m"] = int(rng.choice(m_choices))
        surf, f, delta = build_request(s)
        out.append((surf.X, surf.w, f, surf.X.copy(), np.array([delta])))
    return out


def submit_retry(srv, *args, tries=2000):
    for _ in range(tries):
        try:
            return sk.serve_submit(srv, *args)
        except sk.SkError as e:
            if e.code != sk.SK_EBUSY:
                raise
            time.sleep(0.001)
    raise TimeoutError("server stayed busy")


def test_served_results_match_standalone_bitwise(ctx):
    reqs = mixed_requests(16)
    refs = [sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *r) for r in reqs]
    srv = sk.serve_create(ctx, max_slots=6)
    try:
        tickets = [submit_retry(srv, *r) for r in reqs]
        for t, r, ref in zip(tickets, reqs, refs):
            code, u, st = sk.serve_poll(srv, t, r[3].shape[0], timeout_us=30_000_000)
            assert code == sk.SK_OK
            assert np.array_equal(u, ref)
            assert st["interactions"] == r[3].shape[0] * np.count_nonzero(r[1])
            assert st["submit_us"] <= st["admit_us"] <= st["publish_us"] <= st["done_us"] \
                <= st["ready_us"]
    finally:
        sk.serve_destroy(srv)
    # and the standalone path itself matches the oracle
    for r, ref in list(zip(reqs, refs))[:3]:
        o = oracle.sl(*r)
        assert np.linalg.norm(ref - o) / np.linalg.norm(o) <= 1e-6


def test_same_result_alone_and_in_the_mix(ctx):
    reqs = mixed_requests(24, seed=43)
    probe = reqs[5]
    srv = sk.serve_create(ctx, max_slots=8)
    try:
        t = submit_retry(srv, *probe)
        code, alone, _ = sk.serve_poll(srv, t, probe[3].shape[0], timeout_us=30_000_000)
        assert code == sk.SK_OK
        tickets = []
        for i, r in enumerate(reqs):
            tickets.append((submit_retry(srv, *r), r))
            if i == 11:
                tickets.append((submit_retry(srv, *probe), probe))
        mixed = None
        for tk, r in tickets:
            code, u, _ = sk.serve_poll(srv, tk, r[3].shape[0], timeout_us=30_000_000)
            assert code == sk.SK_OK
            if r is probe:
                mixed = u
        assert mixed is not None and np.array_equal(mixed, alone)
    finally:
        sk.serve_destroy(srv)


def test_large_request_alone_and_in_the_mix(ctx):
    """Above 131,072 targets the standalone call runs two target pairs per
    lane while the server keeps one: the served result is then the same bit
    for bit alone and in any mix, and within FP32 rounding of the standalone
    call and within the tolerance of the oracle."""
    shape = ci.Ellipsoid(1.0, 0.8, 0.5)
    s = ci.make_surface(shape, 129)
    rng = np.random.default_rng(77)
    f = ci.sh_density(s.x0, rng, lmax=8)
    probes, _ = ci.exterior_probes(shape, 40_000, s.h, rng)
    Y = np.concatenate([s.X, probes])
    big = (s.X, s.w, f, Y, np.array([2 * s.h]))
    assert Y.shape[0] > 131_072
    small = mixed_requests(6, m_choices=(17, 33), seed=79)
    srv = sk.serve_create(ctx, max_slots=4)
    try:
        t = submit_retry(srv, *big)
        code, alone, _ = sk.serve_poll(srv, t, Y.shape[0], timeout_us=60_000_000)
        assert code == sk.SK_OK
        tickets = [(submit_retry(srv, *r), r) for r in small[:3]]
        tickets.append((submit_retry(srv, *big), big))
        tickets += [(submit_retry(srv, *r), r) for r in small[3:]]
        mixed = None
        for tk, r in tickets:
            code, u, _ = sk.serve_poll(srv, tk, r[3].shape[0], timeout_us=60_000_000)
            assert code == sk.SK_OK
            if r is big:
                mixed = u
        assert mixed is not None and np.array_equal(mixed, alone)
    finally:
        sk.serve_destroy(srv)
    ref = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *big)
    assert np.linalg.norm(alone - ref) / np.linalg.norm(ref) <= 1e-7
    pick = np.random.default_rng(78).choice(Y.shape[0], 256, replace=False)
    o = oracle.sl(s.X, s.w, f, Y[pick], 2 * s.h)
    assert np.linalg.norm(alone[pick] - o) / np.linalg.norm(o) <= 1e-6


def test_per_target_delta_requests_match_standalone(ctx):
    """Requests with one delta per target (n_delta = M, e.g. delta* of each
    target's patch) are served like scalar-delta ones: bit for bit the
    standalone result, alone and mixed with scalar-delta requests."""
    rng = np.random.default_rng(71)
    reqs = []
    for r in mixed_requests(6, m_choices=(9, 17, 33), seed=71):
        X, W, F, Y, D = r
        reqs.append((X, W, F, Y, D[0] * rng.uniform(0.5, 2.0, Y.shape[0])))
        reqs.append(r)
    refs = [sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *r) for r in reqs]
    srv = sk.serve_create(ctx, max_slots=4)
    try:
        tickets = [submit_retry(srv, *r) for r in reqs]
        for t, r, ref in zip(tickets, reqs, refs):
            code, u, _ = sk.serve_poll(srv, t, r[3].shape[0], timeout_us=30_000_000)
            assert code == sk.SK_OK
            assert np.array_equal(u, ref)
    finally:
        sk.serve_destroy(srv)
    for r, ref in list(zip(reqs, refs))[:2]:
        o = oracle.sl(*r)
        assert np.linalg.norm(ref - o) / np.linalg.norm(o) <= 1e-6


def test_busy_queue_and_too_large_request(ctx):
    w = ci.rbc_workload()
    s = w.surface
    args = (s.X, s.w, w.f, w.targets, w.delta)
    srv = sk.serve_create(ctx, max_slots=1, queue_capacity=1)
    busy = 0
    tickets = []
    try:
        for _ in range(6):
            try:
                tickets.append(sk.serve_submit(srv, *args))
            except sk.SkError as e:
                assert e.code == sk.SK_EBUSY
                busy += 1
        assert busy > 0
        for t in tickets:
            assert sk.serve_poll(srv, t, w.targets.shape[0], timeout_us=30_000_000)[0] == sk.SK_OK
    finally:
        sk.serve_destroy(srv)
    small = sk.serve_create(ctx, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(sk.SkError) as e:
            sk.serve_submit(small, *args)
        assert e.value.code == sk.SK_ENOMEM
    finally:
        sk.serve_destroy(small)


def test_poll_modes_invalid_requests_and_relaunch(ctx):
    r = mixed_requests(1, m_choices=(17,), seed=47)[0]
    srv = sk.serve_create(ctx, idle_exit_us=2000)
    try:
        assert sk.serve_poll(srv, 123456, 3, timeout_us=0)[0] == sk.SK_EINVAL
        with pytest.raises(sk.SkError) as e:
            sk.serve_submit(srv, r[0], r[1], r[2], r[3], np.array([-1.0]))
        assert e.value.code == sk.SK_EINVAL
        t = sk.serve_submit(srv, *r)
        code = sk.serve_poll(srv, t, r[3].shape[0], timeout_us=0)[0]
        assert code in (sk.SK_EAGAIN, sk.SK_OK)
        if code == sk.SK_EAGAIN:
            assert sk.serve_poll(srv, t, r[3].shape[0], timeout_us=30_000_000)[0] == sk.SK_OK
        time.sleep(0.05)  # the persistent kernel exits when idle ...
        t = sk.serve_submit(srv, *r)  # ... and is relaunched for new work
        code, u, _ = sk.serve_poll(srv, t, r[3].shape[0], timeout_us=30_000_000)
        assert code == sk.SK_OK
        assert np.array_equal(u, sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *r))
    finally:
        sk.serve_destroy(srv)


def test_exits_and_relaunches_racing_with_arrivals(ctx):
    """A 300 us idle limit with arrival gaps of 0-2 ms: the persistent kernel
    leaves and is relaunched many times, often while requests are being
    published. Its CTAs leave together (an exit word), so no request is lost
    or left to a partial kernel, and every result is the standalone one."""
    reqs = mixed_requests(24, m_choices=(9, 17, 33, 49), seed=59)
    refs = [sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *r) for r in reqs]
    rng = np.random.default_rng(59)
    srv = sk.serve_create(ctx, max_slots=4, idle_exit_us=300)
    try:
        tickets = []
        for r in reqs:
            tickets.append(submit_retry(srv, *r))
            time.sleep(float(rng.uniform(0.0, 0.002)))
        for t, r, ref in zip(tickets, reqs, refs):
            code, u, _ = sk.serve_poll(srv, t, r[3].shape[0], timeout_us=30_000_000)
            assert code == sk.SK_OK
            assert np.array_equal(u, ref)
    finally:
        sk.serve_destroy(srv)


def test_destroy_drains_pending_requests(ctx):
    reqs = mixed_requests(8, seed=53)
    srv = sk.serve_create(ctx, max_slots=2)
    for r in reqs:
        submit_retry(srv, *r)
    sk.serve_destroy(srv)  # must finish the work and return
    srv = sk.serve_create(ctx)  # the context can serve again
    sk.serve_destroy(srv)


# ---- resident capsules -------------------------------------------------------
ES, ED = 2.0, 20.0


def make_capsule(ctx, m=17, stretch=(1.04, 0.98, 1.0)):
    """A capsule with a Skalak membrane on the stress-free ellipsoid
    (0.9, 1, 1), started from a stretched shape; delta* per step."""
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    cap = sk.Capsule(ctx, m, ref.X * np.array(stretch), ref.w, delta=None, mu=1.0,
                     precision=sk.SK_FP32C)
    cap.set_membrane(ref.X, ES, ED)
    return cap


def submit_capsule_retry(srv, cap, n, dt, flow, tries=2000):
    for _ in range(tries):
        try:
            return sk.serve_submit_capsule(srv, cap, n, dt, flow)
        except sk.SkError as e:
            if e.code != sk.SK_EBUSY:
                raise
            time.sleep(0.001)
    raise TimeoutError("server stayed busy")


def test_served_capsule_steps_equal_capsule_step_bitwise(ctx):
    """n Euler steps of a resident capsule served through the persistent
    kernel leave the nodes bit for bit where capsule_step leaves an identical
    capsule: each step's membrane force, weights, delta* and update are the
    same operations, and each step's sum is the standalone one. The capsule's
    state stays on the device across two requests."""
    flow = (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0)
    a, b = make_capsule(ctx), make_capsule(ctx)
    srv = sk.serve_create(ctx, max_slots=4)
    try:
        a.step(4, 1e-3, None, flow)
        a.step(3, 1e-3, None, flow)
        t = submit_capsule_retry(srv, b, 4, 1e-3, flow)
        code, x4, st = sk.serve_poll(srv, t, b.N, timeout_us=60_000_000)
        assert code == sk.SK_OK
        assert st["interactions"] == 4 * b.N * np.count_nonzero(make_surface_w(17))
        t = submit_capsule_retry(srv, b, 3, 1e-3, flow)
        code, x7, _ = sk.serve_poll(srv, t, b.N, timeout_us=60_000_000)
        assert code == sk.SK_OK
    finally:
        sk.serve_destroy(srv)
    assert np.array_equal(x7, a.positions())
    assert np.array_equal(x7, b.positions())
    assert not np.array_equal(x4, x7)
    a.close()
    b.close()


def make_surface_w(m):
    return ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m).w


def test_shear_rate_sweep_in_the_mix(ctx):
    """A parameter sweep: capsules at four shear rates and a Poiseuille flow,
    each a multi-step request, served together with ordinary single-layer
    requests; every capsule ends where capsule_step takes its twin, and every
    ordinary request equals its standalone result, bit for bit."""
    flows = [(sk.SK_FLOW_SHEAR, r, 0.0, 0.0) for r in (0.5, 1.0, 2.0, 4.0)] + \
            [(sk.SK_FLOW_POISEUILLE, 0.0, 1.0, 5.0)]
    twins = [make_capsule(ctx, m=13 + 4 * (i % 2)) for i in range(len(flows))]
    served = [make_capsule(ctx, m=13 + 4 * (i % 2)) for i in range(len(flows))]
    for cap, fl in zip(twins, flows):
        cap.step(5, 1e-3, None, fl)
    reqs = mixed_requests(10, seed=47)
    refs = [sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_HOST, *r) for r in reqs]
    srv = sk.serve_create(ctx, max_slots=8)
    try:
        tickets = []
        for i in range(max(len(flows), len(reqs))):
            if i < len(flows):
                tickets.append(("cap", i, submit_capsule_retry(srv, served[i], 5, 1e-3, flows[i])))
            if i < len(reqs):
                tickets.append(("req", i, submit_retry(srv, *reqs[i])))
        for kind, i, t in tickets:
            n = served[i].N if kind == "cap" else reqs[i][3].shape[0]
            code, u, _ = sk.serve_poll(srv, t, n, timeout_us=60_000_000)
            assert code == sk.SK_OK
            if kind == "cap":
                assert np.array_equal(u, twins[i].positions()), i
            else:
                assert np.array_equal(u, refs[i]), i
    finally:
        sk.serve_destroy(srv)
    for c in twins + served:
        c.close()


def test_capsule_request_errors(ctx):
    cap = make_capsule(ctx, m=9)
    fp64 = sk.Capsule(ctx, 9, ci.make_surface(ci.Sphere(1.0), 9).X,
                      ci.make_surface(ci.Sphere(1.0), 9).w, precision=sk.SK_FP64)
    srv = sk.serve_create(ctx, max_slots=2)
    try:
        with pytest.raises(sk.SkError) as e:
            sk.serve_submit_capsule(srv, fp64, 1, 1e-3)
        assert e.value.code == sk.SK_EINVAL
        with pytest.raises(sk.SkError) as e:
            sk.serve_submit_capsule(srv, cap, 0, 1e-3)
        assert e.value.code == sk.SK_EINVAL
        t = sk.serve_submit_capsule(srv, cap, 50, 1e-3)
        with pytest.raises(sk.SkError) as e:   # one request per capsule at a time
            sk.serve_submit_capsule(srv, cap, 1, 1e-3)
        assert e.value.code == sk.SK_EBUSY
        code, _, _ = sk.serve_poll(srv, t, cap.N, timeout_us=60_000_000)
        assert code == sk.SK_OK
        t = sk.serve_submit_capsule(srv, cap, 1, 1e-3)   # free again
        assert sk.serve_poll(srv, t, cap.N, timeout_us=60_000_000)[0] == sk.SK_OK
    finally:
        sk.serve_destroy(srv)
    cap.close()
    fp64.close()
