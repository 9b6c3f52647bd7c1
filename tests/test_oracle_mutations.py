"""Planted mistakes in a copy of the oracle must fail at least one pin.

Each case rewrites one expression of stokes_oracle.c (a dropped or altered
term, a wrong sign, a swapped operand, a wrong index), compiles the copy into
a temporary library and runs the pin battery against it. This shows that the
pins constrain every part of the oracle's arithmetic, not just its output on
one input. The real oracle is never modified.
"""

import os

import numpy as np
import pytest

import oracle
import oracle_pins as P

MUTATIONS = {
    "s1 polynomial": ("(2.0 * p * p - 5.0)", "(2.0 * p * p - 4.0)"),
    "s2 polynomial": ("- 14.0 * p2 + 3.0)", "- 13.0 * p2 + 3.0)"),
    "s3 polynomial": ("- 36.0 * p2 * p2 + 6.0 * p2", "- 36.0 * p2 * p2 + 5.0 * p2"),
    "s1 series term": ("- 5.0 * exp_coef(n)) / 3.0;", "- 4.0 * exp_coef(n)) / 3.0;"),
    "s2 series term": ("+ 3.0 * exp_coef(n)) / 3.0;", "+ 2.0 * exp_coef(n)) / 3.0;"),
    "s3 series shift": ("c3[n] = a3[n + 2];", "c3[n] = a3[n + 1];"),
    "rr term sign": ("f0 * a + fd * d0 * b", "f0 * a - fd * d0 * b"),
    "rr term dropped": ("wp * (f2 * a + fd * d2 * b)", "wp * (f2 * a)"),
    "transposed rr term": ("wp * (f1 * a + fd * d1 * b)", "wp * (f1 * a + fd * f1 * b)"),
    "viscosity dropped": ("1.0 / (8.0 * ORACLE_PI * mu)", "1.0 / (8.0 * ORACLE_PI)"),
    "delta of source": ("const double dl = delta[n_delta == 1 ? 0 : t];\n    const double x0",
                        "const double dl = delta[0];\n    const double x0"),
    "delta cubed": ("oracle_k(2, 0, p) / (dl * dl * dl)", "oracle_k(2, 0, p) / (dl * dl)"),
    "stresslet sign": ("w[j] * pref * (-6.0)", "w[j] * pref * (6.0)"),
    "stresslet normal swapped": ("d0 * nrm[3 * j] + d1 * nrm[3 * j + 1] + d2 * nrm[3 * j + 2]",
                                 "d0 * q[3 * j] + d1 * q[3 * j + 1] + d2 * q[3 * j + 2]"),
    "series switch": ("#define SERIES_SWITCH 1.0", "#define SERIES_SWITCH 0.0"),
}


def _run_battery(orc):
    failed = []
    for pin in P.SL_PINS + P.DL_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(orc)
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mutated = tmp_path / "mutated.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.compile_library(str(mutated), str(tmp_path / "libmutated.so"))
    failed = _run_battery(oracle.Oracle(lib))
    assert failed, f"no pin caught the planted mistake '{name}'"


def test_unmutated_oracle_passes_battery():
    assert _run_battery(oracle.default()) == []
