"""Host logic of the work decomposition (paper_2310_13908_gb300/csrc/sk_decomp.h):
how many source chunks split each target block's sum, the FP64 kernel's CTA
size, and whether the FP32C pair kernel finishes its target blocks itself.
The header is compiled with the host C++ compiler against the CUDA headers
and driven over measured shapes and sweeps; no GPU is involved."""

import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_13908_gb300", "csrc")
SMS = 152  # GB300

PROGRAM = r"""
#include <cstdio>
#include "sk_decomp.h"
// stdin: "precision N M sm_count" per line; stdout: "n_chunks threads64 fuse_finish np"
int main() {
  int prec, sm;
  long long N, M;
  while (std::scanf("%d %lld %lld %d", &prec, &N, &M, &sm) == 4) {
    sk::EvalShape s;
    s.precision = prec;
    s.N = N;
    s.M = M;
    sk::choose_decomposition(s, sm);
    std::printf("%d %d %d %d\n", s.n_chunks, s.threads64, s.fuse_finish ? 1 : 0,
                sk::pair32_np(M));
  }
  return 0;
}
"""

FP64, FP32C = 0, 1   # SK_FP64, SK_FP32C of include/stokesreg.h


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        inc = os.path.join(base, "include")
        if base and os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def decompose(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    d = tmp_path_factory.mktemp("decomp")
    (d / "program.cpp").write_text(PROGRAM)
    exe = d / "program"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, str(d / "program.cpp"), "-o",
                    str(exe)], check=True)

    def run(cases):
        text = "".join(f"{p} {n} {m} {sm}\n" for p, n, m, sm in cases)
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True,
                             check=True).stdout.split("\n")
        return [tuple(int(v) for v in line.split()) for line in out if line.strip()]
    return run


def _blocks(M, np_):
    tgt_cta = 256 * 2 * np_
    return -(-max(M, 1) // tgt_cta)


def test_measured_shapes(decompose):
    # ellipsoid m = 257 + 100k probes (the benchmark step): the profiled grid of
    # 482 target blocks x 22 chunks = 10604 CTAs, finishing fused
    c3, c2, c1_64, c1_32 = decompose([(FP32C, 393216, 493216, SMS), (FP32C, 24576, 24576, SMS),
                                      (FP64, 1944, 1944, SMS), (FP32C, 1944, 1944, SMS)])
    assert c3 == (22, 256, 1, 2) and _blocks(493216, 2) * 22 == 10604
    # the cell at m = 65: 48 target blocks, separate finish kernels; too small
    # for 32 full waves, so the most chunks (64: measured fastest)
    assert c2[2] == 0 and _blocks(24576, 1) == 48 and c2[3] == 1 and c2[0] == 64
    # the sphere at m = 19 in FP64: 64-thread CTAs, one 128-source tile per chunk
    assert c1_64[1] == 64 and c1_64[0] == math.ceil(1944 / 128)
    assert c1_32[2] == 0


def test_fused_finish_from_two_blocks_per_sm(decompose):
    # NP = 2 (1024 targets per block) above 131072 targets
    Ms = [2 * SMS * 1024 - 1024, 2 * SMS * 1024 - 1023, 2 * SMS * 1024, 2 * SMS * 1024 + 1]
    got = decompose([(FP32C, 200000, M, SMS) for M in Ms])
    for M, (_, _, fused, np_) in zip(Ms, got):
        assert np_ == 2
        assert fused == int(_blocks(M, 2) >= 2 * SMS), (M, fused)
    assert [g[2] for g in got] == [0, 1, 1, 1]
    # below the NP switch no grid reaches 2 blocks per SM (256 blocks at most)
    assert all(g[2] == 0 for g in decompose([(FP32C, 10 ** 6, M, SMS) for M in
                                              (1, 512, 131072)]))


def test_pairs_per_lane_switch_at_131072_targets(decompose):
    got = decompose([(FP32C, 50000, M, SMS) for M in (131071, 131072, 131073)])
    assert [g[3] for g in got] == [1, 1, 2]


def test_chunk_counts_fill_waves(decompose):
    cases = []
    for N in (0, 1, 300, 5000, 24576, 98304, 393216, 2_000_000):
        for M in (1, 700, 24576, 131072, 131073, 493216, 2_000_000):
            cases.append((FP32C, N, M, SMS))
    for (p, N, M, sm), (nc, t64, fused, np_) in zip(cases, decompose(cases)):
        tiles = -(-max(N, 1) // 256)
        many = max(1, min(64, tiles))
        assert 1 <= nc <= many, (N, M, nc)
        slots = sm * (2 if np_ == 2 else 3)
        waves = _blocks(M, np_) * nc / slots
        cap = max(1, min(64, tiles // 2))
        # enough work: at least 32 waves, the last one at least 98% full
        if _blocks(M, np_) * cap / slots >= 40:
            assert waves >= 32 and waves / math.ceil(waves) >= 0.98, (N, M, nc, waves)
        # too little for 32 waves: the most chunks, down to one tile each
        if _blocks(M, np_) * cap / slots < 32:
            assert nc == many, (N, M, nc)
        assert t64 == 256  # the FP64 CTA size is not touched on the FP32C path


def test_fp64_small_problems_take_64_thread_ctas(decompose):
    cases = [(FP64, N, M, SMS) for N, M in ((1944, 1944), (24576, 24576), (393216, 493216),
                                            (100, 100), (0, 5))]
    got = decompose(cases)
    for (p, N, M, sm), (nc, t64, fused, _) in zip(cases, got):
        assert fused == 0
        if t64 == 64:
            assert nc == min(64, -(-max(N, 1) // 128))
        else:
            # 512 targets per 256-thread CTA fill four waves of two CTAs per SM
            assert t64 == 256 and _blocks(M, 1) * nc >= 4 * 2 * sm
    assert got[0][1] == 64 and got[2][1] == 256
