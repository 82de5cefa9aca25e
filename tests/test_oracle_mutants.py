"""The pins catch plausible mistakes in the oracle.

Each case copies the oracle's C source to a temporary directory, plants one
mistake by a textual substitution (a dropped sticky bit, ties away from zero,
an exponent off by one, a wrong signed-zero rule, a dropped hidden bit, a
subnormal treated as normal), builds that copy, and checks that at least one
pin -- closed forms, math.fsum, the IEEE bracketing definition -- now fails.
The committed oracle itself is never modified.  CPU only.
"""
from __future__ import annotations

import ctypes
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from paper_1605_05436_gb300 import workloads as W
from tests import fpref
from tests.test_oracle_pins import CLOSED, encode_inputs, expected_matches

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "exactsum_oracle.c")

MUTANTS = {
    "no_sticky": ("int sticky = or_any_below(M, shift - 1);", "int sticky = 0;"),
    "ties_away": ("if (mode == OR_RNE) round_up = half && (sticky || (q & 1));",
                  "if (mode == OR_RNE) round_up = half;"),
    "exponent_off_by_one": ("int p = (E == 0) ? 0 : (int)E - 1;", "int p = (E == 0) ? 0 : (int)E;"),
    "zero_sign_rdown": ("return mode == OR_RDOWN ? neg_zero : 0;", "return 0;"),
    "no_hidden_bit": ("uint64_t m = (E == 0) ? F : (F | ((uint64_t)1 << f.frac_bits));", "uint64_t m = F;"),
    "subnormal_as_normal": ("uint64_t m = (E == 0) ? F : (F | ((uint64_t)1 << f.frac_bits));",
                            "uint64_t m = F | ((uint64_t)1 << f.frac_bits);"),
    "overflow_rtz_to_inf": ("else if (mode == OR_RTZ) to_inf = 0;", "else if (mode == OR_RTZ) to_inf = 1;"),
    "negative_as_positive": ("if (sign) or_sub_shifted(&s->sum, m, p);", "if (0) or_sub_shifted(&s->sum, m, p);"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    d = tmp_path / name
    d.mkdir()
    src = d / "oracle.c"
    src.write_text(text.replace(old, new))
    lib = d / "liboracle.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", "-o", str(lib), str(src)])
    h = ctypes.CDLL(str(lib))
    h.oracle_sum.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int, ctypes.c_void_p]
    h.oracle_sum.restype = ctypes.c_int

    def exact_sum(bits, i, o, m):
        a = np.ascontiguousarray(bits)
        res = np.zeros(1, dtype=fpref.NP_BITS[o])
        assert h.oracle_sum(a.ctypes.data if a.size else None, a.size, i, o, m, 1, res.ctypes.data) == 0
        return int(res[0])

    return exact_sum


def pins_fail(exact_sum) -> bool:
    """True if at least one pin rejects this oracle."""
    for name, i, o, m, inputs, expected, why in CLOSED:
        if not expected_matches(expected, exact_sum(encode_inputs(inputs, i), i, o, m), o):
            return True
    rng = np.random.default_rng(0)
    for seed in range(3):
        x = rng.uniform(-1, 1, 500)
        if exact_sum(x.view(np.uint64), 0, 0, 0) != fpref.from_float(math.fsum(x.tolist()), 0):
            return True
    for dt, bits in ((1, W.wide_f32(300, seed=1, subnormal_frac=0.2)), (2, W.wide_bf16(300, seed=2))):
        S = fpref.exact(bits, dt)
        for mode in range(4):
            try:
                fpref.check_rounding(S, exact_sum(bits, dt, dt, mode), dt, mode)
            except AssertionError:
                return True
    return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    assert pins_fail(build_mutant(tmp_path, name)), f"no pin catches the '{name}' mistake"


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_unmutated_copy_passes_pins(tmp_path):
    """Control: the same harness on an unchanged copy finds nothing."""
    MUTANTS["identity"] = ("#define OR_LIMBS 96", "#define OR_LIMBS 96")
    try:
        assert not pins_fail(build_mutant(tmp_path, "identity"))
    finally:
        del MUTANTS["identity"]
