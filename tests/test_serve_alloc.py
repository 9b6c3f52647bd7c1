"""Host logic of serving admission: the first-fit range allocator of the
request arena and the staging pool (paper_2310_13908_gb300/csrc/sk_range_alloc.h),
compiled with the host C++ compiler and driven by random alloc/release
sequences against an independent model: a bitmap of 256-byte units in which
first fit is the lowest offset that starts enough consecutive free units."""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2310_13908_gb300", "csrc", "sk_range_alloc.h")
UNIT = 256

PROGRAM = r"""
#include <cstdio>
#include "sk_range_alloc.h"
// stdin: "Z size" reset, "A n" alloc (prints offset or -1), "R off n" release,
// "F" prints the free ranges as "off:len ..." on one line
int main() {
  sk::RangeAlloc a;
  char op;
  while (std::scanf(" %c", &op) == 1) {
    unsigned long long x = 0, y = 0;
    if (op == 'Z') { std::scanf("%llu", &x); a.reset(x); }
    else if (op == 'A') {
      std::scanf("%llu", &x);
      size_t off = 0;
      if (a.alloc(x, &off)) std::printf("%llu\n", (unsigned long long)off);
      else std::printf("-1\n");
    } else if (op == 'R') { std::scanf("%llu %llu", &x, &y); a.release(x, y); }
    else if (op == 'F') {
      for (const auto& kv : a.free_ranges())
        std::printf("%llu:%llu ", (unsigned long long)kv.first, (unsigned long long)kv.second);
      std::printf("\n");
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("range_alloc")
    src = d / "program.cpp"
    src.write_text(PROGRAM)
    exe = d / "program"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.dirname(HEADER), str(src), "-o",
                    str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout
        return out.splitlines()
    return run


class BitmapModel:
    def __init__(self, size):
        assert size % UNIT == 0
        self.free = np.ones(size // UNIT, dtype=bool)

    def alloc(self, n):
        k = max(1, -(-n // UNIT))
        run = 0
        for i, f in enumerate(self.free):
            run = run + 1 if f else 0
            if run == k:
                start = i - k + 1
                self.free[start:i + 1] = False
                return start * UNIT
        return -1

    def release(self, off, n):
        k = max(1, -(-n // UNIT))
        assert not self.free[off // UNIT: off // UNIT + k].any()
        self.free[off // UNIT: off // UNIT + k] = True

    def ranges(self):
        out, i = [], 0
        while i < len(self.free):
            if self.free[i]:
                j = i
                while j < len(self.free) and self.free[j]:
                    j += 1
                out.append((i * UNIT, (j - i) * UNIT))
                i = j
            else:
                i += 1
        return out


def _parse_ranges(line):
    return [tuple(int(v) for v in tok.split(":")) for tok in line.split()]


def test_first_fit_offsets_and_coalescing(program):
    out = program(["Z 4096", "A 1", "A 256", "A 257", "A 0", "F", "R 256 256", "A 300", "A 200",
                  "F", "R 0 1", "R 1024 1", "R 512 257", "F", "A 4096", "A 1"])
    # 1 and 256 bytes take one unit each, 257 takes two, 0 takes one
    assert out[:4] == ["0", "256", "512", "1024"]
    assert _parse_ranges(out[4]) == [(1280, 2816)]
    # the freed unit at 256 is too small for 300 bytes, then exactly fits 200
    assert out[5:7] == ["1280", "256"]
    assert _parse_ranges(out[7]) == [(1792, 2304)]
    # releases merge with both neighbours
    assert _parse_ranges(out[8]) == [(0, 256), (512, 768), (1792, 2304)]
    assert out[9:] == ["-1", "0"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_sequences_match_the_bitmap_model(program, seed):
    rng = np.random.default_rng(seed)
    size = 64 * UNIT
    model = BitmapModel(size)
    cmds, expect, live = [f"Z {size}"], [], []
    for _ in range(600):
        if live and rng.random() < 0.45:
            off, n = live.pop(int(rng.integers(len(live))))
            model.release(off, n)
            cmds.append(f"R {off} {n}")
        else:
            n = int(rng.choice([0, 1, 255, 256, 257, 700, 2048, 5000]))
            off = model.alloc(n)
            cmds.append(f"A {n}")
            expect.append(str(off))
            if off >= 0:
                live.append((off, n))
        if rng.random() < 0.1:
            cmds.append("F")
            expect.append(model.ranges())
    got = program(cmds)
    assert len(got) == len(expect)
    for g, e in zip(got, expect):
        if isinstance(e, list):
            assert _parse_ranges(g) == e
        else:
            assert g == e
    # releasing every live block restores the whole range
    for off, n in live:
        cmds.append(f"R {off} {n}")
    assert _parse_ranges(program(cmds + ["F"])[-1]) == [(0, size)]
