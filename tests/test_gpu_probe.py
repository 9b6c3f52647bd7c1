"""Microbenchmark probes of the throughput ceilings (needs a GB300): the
values are positive and within plausible bounds of the part's unit counts
(152 SMs x 128 FP32 lanes x ~2 GHz; FP64 about 1/64 of FP32)."""

import pytest

sk = pytest.importorskip("paper_2310_13908_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_probe_peaks_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with sk.Context(0) as c:
        p = sk.sk_probe_peaks(c.handle)
    sms = p["sm_count"]
    assert sms > 0
    fp32_nominal = 2 * 128 * sms * 2.2e9 / 1e12   # above any SM clock of the part
    assert 0.3 * fp32_nominal < p["ffma2_tflops"] < 1.05 * fp32_nominal, p
    assert 0.05 < p["dfma_tflops"] < 0.1 * fp32_nominal, p
    # a far pair costs 17 FMA-pipe lane operations: at most the FFMA2 rate / 17
    ceiling = p["ffma2_tflops"] * 1e12 / 2 / 17
    assert 0.3 * ceiling < p["far_pairs_per_s"] < 1.05 * ceiling, p
