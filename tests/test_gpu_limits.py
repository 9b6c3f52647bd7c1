"""Size limits of the C ABI at the top of the source range (needs a GB300).

SK_FP32C names a near pair by its source's original index in 25 bits, so
stokes_sl_eval and stokes_dl_eval take at most 2^25 nodes in that precision.
At exactly 2^25 nodes every near pair must still reach the right node,
including the nodes whose index sets bit 24; one node more is rejected with
SK_EINVAL before any work is enqueued. SK_FP64 keeps no such list and is
checked at the same size.

Inputs: 2^25 seeded random nodes on the unit sphere with equal weights
4 pi / N, a random density, delta = 2h with h = sqrt(4 pi / N). The targets are
nodes at the extremes of the index range and at random indices (each has the
r = 0 pair of Sec. 3.4 and a few more pairs inside rho_T delta), plus exterior
points 0.1h-5h off the surface. Both layers in both precisions are compared with
the FP64 oracle on every target.
"""

import numpy as np
import pytest

import oracle

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N_MAX = 1 << 25
TOL = {sk.SK_FP64: 1e-12, sk.SK_FP32C: 1e-6}
ELEM = {sk.SK_FP64: 1e-12, sk.SK_FP32C: 1e-5}


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = sk.Context(0)
    yield c.handle
    c.close()


@pytest.fixture(scope="module")
def top_range():
    rng = np.random.default_rng(2525)
    X = rng.standard_normal((N_MAX, 3))
    X /= np.linalg.norm(X, axis=1)[:, None]
    w = np.full(N_MAX, 4.0 * np.pi / N_MAX)
    f = rng.standard_normal((N_MAX, 3))
    h = np.sqrt(4.0 * np.pi / N_MAX)
    edge = [0, 1, (1 << 24) - 1, 1 << 24, (1 << 24) + 1, N_MAX - 2, N_MAX - 1]
    picks = np.concatenate([edge, rng.choice(N_MAX, 41, replace=False)])
    on = X[picks]
    d = rng.standard_normal((16, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    off = d * (1.0 + h * rng.uniform(0.1, 5.0, 16))[:, None]
    Y = np.concatenate([on, off])
    delta = np.array([2.0 * h])
    ref_sl = oracle.sl(X, w, f, Y, delta, 1.0)
    # the unit sphere's normal is X itself; f serves as the double layer density
    ref_dl = oracle.dl(X, w, X, f, Y, delta)
    return X, w, f, Y, delta, ref_sl, ref_dl


@pytest.mark.parametrize("layer", ["sl", "dl"])
@pytest.mark.parametrize("prec", [sk.SK_FP32C, sk.SK_FP64])
def test_at_max_sources(ctx, top_range, prec, layer):
    X, w, f, Y, delta, ref_sl, ref_dl = top_range
    dev = lambda a: torch.as_tensor(a, device="cuda")
    if layer == "sl":
        ref = ref_sl
        u = sk.stokes_sl_eval(ctx, prec, sk.SK_DEVICE, dev(X), dev(w), dev(f), dev(Y),
                              dev(delta), 1.0)
    else:
        ref = ref_dl
        u = sk.stokes_dl_eval(ctx, prec, sk.SK_DEVICE, dev(X), dev(w), dev(X), dev(f), dev(Y),
                              dev(delta))
    u = u.cpu().numpy()
    assert np.all(np.isfinite(u))
    e = rel_l2(u, ref)
    # every target, as in the parity tests: a near pair paired with the wrong
    # node would leave an error of the order of that pair's term
    scale = np.abs(ref).max()
    err = np.abs(u - ref).max(axis=1) / scale
    print(f"{layer} prec {prec}: rel-L2 {e:.3e}, max element {err.max():.3e} (of max|u|), "
          f"index extremes {np.array2string(err[:7], precision=2)}")
    assert e <= TOL[prec], f"rel-L2 {e:.3e} at N = 2^25"
    assert err.max() <= ELEM[prec], f"max element error {err.max():.3e} (of max|u|)"


def test_fp32c_rejects_one_node_more(ctx):
    n = N_MAX + 1
    X = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    Y = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    d = torch.ones(1, dtype=torch.float64, device="cuda")
    u = torch.full((4, 3), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkError) as e:
        sk.stokes_sl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, X, w, X, Y, d, 1.0, u_out=u)
    assert e.value.code == sk.SK_EINVAL
    with pytest.raises(sk.SkError) as e:
        sk.stokes_dl_eval(ctx, sk.SK_FP32C, sk.SK_DEVICE, X, w, X, X, Y, d, u_out=u)
    assert e.value.code == sk.SK_EINVAL
    # rejected before any work: the output is untouched
    assert torch.all(u == 7.0)
