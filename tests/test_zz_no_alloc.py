"""stokes_sl_eval_noalloc: the single layer for callers that cannot allocate.

Callers running under a framework-owned memory budget, or in loops where a
cudaMalloc/cudaFree would stall the device, cannot let the library allocate.
The no-allocation entry point works in a static device scratch array inside
the library instead of a context workspace. These tests call it through the
C ABI twice in a row, on two different problems, and compare each result with
stokes_sl_eval (SK_FP32C, device memory) within the FP32C tolerance of the
parity tests, and with the FP64 oracle. Where the scratch holds the context
call's split of the source sum (the 1944-node sphere), the two calls must
agree bit for bit, as the header states. The file is collected last so that
a stopping run has already run every other test; it also passes alone in a
fresh process.
"""

import numpy as np
import pytest

import capsule_inputs as ci
import oracle

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = sk.Context(0)
    yield c.handle
    c.close()


def test_noalloc_matches_context_entry_point_twice_in_a_row(ctx):
    # N = 1944 (its scratch holds the context's split: bitwise), then 24,576
    problems = [(ci.sphere_noise_workload(), True), (ci.rbc_workload(), False)]
    for w, bitwise in problems:
        s = w.surface
        args = [_dev(a) for a in (s.X, s.w, w.f, w.targets, w.delta)]
        ref = sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, *args, w.mu).cpu().numpy()
        u = sk.stokes_sl_eval_noalloc(*args, w.mu).cpu().numpy()
        assert np.all(np.isfinite(u))
        if bitwise:
            assert np.array_equal(u, ref)
        assert _rel_l2(u, ref) <= 1e-6
        assert np.abs(u - ref).max() <= 1e-5 * np.abs(ref).max()
        # and against the FP64 oracle on sampled targets, at the FP32C tolerance
        idx = np.random.default_rng(5).choice(w.targets.shape[0], 256, replace=False)
        exact = oracle.sl(s.X, s.w, w.f, w.targets[idx], w.delta, w.mu)
        assert _rel_l2(u[idx], exact) <= 1e-6


def test_noalloc_rejects_problems_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 200_000
    X = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    W = torch.ones(n, dtype=torch.float64, device="cuda")
    D = torch.full((1,), 0.1, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval_noalloc(X, W, X, X, D, 1.0)
    assert e.value.code == sk.SK_EINVAL
