"""Pins for the CPU oracle: checks against things other than the oracle.

- hand-derived closed forms (tests/golden/closed_forms.txt);
- ``math.fsum`` (a correctly rounded FP64 sum of finite inputs) and
  ``float(Fraction)`` (correct FP64 rounding of an exact rational);
- the IEEE definition of every rounding mode, checked by bracketing the exact
  rational sum between numpy ``nextafter`` neighbours (fpref.check_rounding);
- the set-equality construction from the proof of the Section 3 lower bound;
- the structure of the cancelling workload (the exact sum equals the sum of
  the residue alone);
- invariants: permutation, negation, scaling by powers of two, splitting;
- brute force over every short sequence from a small value grid.
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1605_05436_gb300 import workloads as W
from tests import fpref
from tests.fpref import F64, F32, BF16, RNE, RTZ, RUP, RDOWN

HERE = os.path.dirname(os.path.abspath(__file__))
DT = {"f64": F64, "f32": F32, "bf16": BF16}
MODE = {"rne": RNE, "rtz": RTZ, "rup": RUP, "rdown": RDOWN}


def load_closed_forms():
    cases = []
    with open(os.path.join(HERE, "golden", "closed_forms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, i, o, m, inputs, expected, why = [f.strip() for f in line.split("|")]
            cases.append((name, DT[i], DT[o], MODE[m], inputs, expected, why))
    return cases


def parse_value(tok: str) -> float:
    tok = tok.strip()
    if tok in ("inf", "+inf"):
        return math.inf
    if tok == "-inf":
        return -math.inf
    if tok == "nan":
        return math.nan
    return float.fromhex(tok)


def encode_inputs(inputs: str, dtype: int) -> np.ndarray:
    vals = [parse_value(t) for t in inputs.split(",") if t.strip()]
    bits = [fpref.from_float(v, dtype) for v in vals]
    return np.array(bits, dtype=fpref.NP_BITS[dtype])


def expected_matches(expected: str, r: int, out: int) -> bool:
    if expected == "nan":
        return fpref.is_nan(r, out)
    if expected == "+0":
        return r == 0
    if expected == "-0":
        return r == fpref.SIGN_BIT[out]
    return r == fpref.from_float(parse_value(expected), out)


CLOSED = load_closed_forms()


@pytest.mark.parametrize("case", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(case):
    name, i, o, m, inputs, expected, why = case
    x = encode_inputs(inputs, i)
    r = oracle.exact_sum(x, i, o, m)
    assert expected_matches(expected, r, o), f"{name}: got {r:#x} ({why})"
    # the same with several threads and reversed order
    r2 = oracle.exact_sum(x[::-1].copy(), i, o, m, threads=3)
    assert r2 == r or (expected == "nan" and fpref.is_nan(r2, o))


def test_nan_is_canonical_quiet():
    x = np.array([0x7FF0000000000001, 0x3FF0000000000000], dtype=np.uint64)  # signalling NaN
    assert oracle.exact_sum(x) == 0x7FF8000000000000
    x = np.array([0xFFF8000000000123], dtype=np.uint64)
    assert oracle.exact_sum(x, F64, F32) == 0x7FC00000
    x = np.array([0xFFC1], dtype=np.uint16)
    assert oracle.exact_sum(x, BF16, BF16) == 0x7FC0


@pytest.mark.parametrize("seed", range(6))
def test_fsum_uniform(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 5000))
    x = rng.uniform(-1, 1, n)
    r = oracle.exact_sum(x.view(np.uint64), threads=1 + seed % 4)
    assert r == fpref.from_float(math.fsum(x.tolist()), F64)


@pytest.mark.parametrize("seed", range(6))
def test_fsum_wide_exponents(seed):
    rng = np.random.default_rng(100 + seed)
    n = 3000
    bits = W._random_f64_bits(rng, n, -1000, 1000)
    x = bits.view(np.float64)
    r = oracle.exact_sum(bits, threads=2)
    assert r == fpref.from_float(math.fsum(x.tolist()), F64)


def test_fsum_cancelling_small():
    # the cancelling workload at a small size: pairs cancel, the residue remains
    n = (1 << 14) + 1024
    bits = W.cancelling_f64(n, seed=3)
    x = bits.view(np.float64)
    r = oracle.exact_sum(bits, threads=4)
    assert r == fpref.from_float(math.fsum(x.tolist()), F64)
    res = W.cancelling_residue(n, seed=3)
    assert r == fpref.from_float(math.fsum(res.view(np.float64).tolist()), F64)
    assert oracle.exact_value(bits) == oracle.exact_value(res)


@pytest.mark.parametrize("dtype", [F64, F32, BF16])
@pytest.mark.parametrize("mode", [RNE, RTZ, RUP, RDOWN])
def test_exact_value_and_modes_bracket(dtype, mode):
    rng = np.random.default_rng(7 + dtype * 4 + mode)
    if dtype == F64:
        bits = W._random_f64_bits(rng, 400, -60, 60)
    elif dtype == F32:
        bits = W.wide_f32(400, seed=int(rng.integers(1 << 30)), subnormal_frac=0.1)
    else:
        bits = W.wide_bf16(400, seed=int(rng.integers(1 << 30)))
    S = fpref.exact(bits, dtype)
    unit = {F64: -1074, F32: -149, BF16: -133}[dtype]
    assert Fraction(oracle.exact_value(bits, dtype)) * Fraction(2) ** unit == S
    for out in (F64, F32, BF16):
        r = oracle.exact_sum(bits, dtype, out, mode, threads=2)
        if S == 0:
            continue
        fpref.check_rounding(S, r, out, mode)


def test_round_value_against_fraction():
    rng = np.random.default_rng(11)
    for _ in range(300):
        e = int(rng.integers(-1200, 1100))
        v = int(rng.integers(1, 1 << 62)) * (1 if rng.random() < 0.5 else -1)
        S = Fraction(v) * Fraction(2) ** e
        r = oracle.round_value(v, e, F64, RNE)
        try:
            want = float(S)
        except OverflowError:
            want = math.copysign(math.inf, v)
        assert r == fpref.from_float(want, F64), (v, e)
        for out in (F32, BF16):
            for mode in (RNE, RTZ, RUP, RDOWN):
                fpref.check_rounding(S, oracle.round_value(v, e, out, mode), out, mode)


def test_set_equality_construction():
    """Proof of the Section 3 lower bound: numbers -2^(tau c_i) and +2^(tau d_i),
    tau a power of two above log2 n, sum to zero iff C == D as multisets."""
    rng = np.random.default_rng(5)
    n = 200
    tau = 8  # > log2(400)
    C = rng.integers(-120, 120, n)
    D = rng.permutation(C)
    vals = [-math.ldexp(1.0, tau * int(c)) for c in C] + [math.ldexp(1.0, tau * int(d)) for d in D]
    vals = [v for v in vals]
    bits = np.array(vals).view(np.uint64)
    assert oracle.exact_sum(bits) == 0
    # change one element of D: the sum is exactly 2^(tau d') - 2^(tau d)
    D2 = D.copy()
    D2[17] = D[17] + 1
    vals2 = [-math.ldexp(1.0, tau * int(c)) for c in C] + [math.ldexp(1.0, tau * int(d)) for d in D2]
    r = oracle.exact_sum(np.array(vals2).view(np.uint64))
    want = math.ldexp(1.0, tau * int(D2[17])) - math.ldexp(1.0, tau * int(D[17]))
    assert r == fpref.from_float(want, F64)


def test_invariants():
    rng = np.random.default_rng(9)
    bits = W.cancelling_f64(4096 + 64, seed=9, residue=64, emin=-300, emax=300)
    x = bits.view(np.float64)
    base = oracle.exact_sum(bits)
    # permutation
    for _ in range(3):
        assert oracle.exact_sum(rng.permutation(bits)) == base
    # negation symmetry (round to nearest)
    neg = (-x).view(np.uint64)
    assert oracle.exact_sum(neg) == base ^ (1 << 63)
    # directed modes swap under negation
    assert oracle.exact_sum(neg, F64, F64, RUP) == oracle.exact_sum(bits, F64, F64, RDOWN) ^ (1 << 63)
    # scaling by 2^k without under/overflow scales the result
    for k in (-20, 7, 300):
        sc = np.ldexp(x, k).view(np.uint64)
        r = fpref.to_float(oracle.exact_sum(sc), F64)
        assert r == math.ldexp(fpref.to_float(base, F64), k)
    # splitting: the exact value of the whole is the sum of the parts
    cut = 1234
    assert oracle.exact_value(bits) == oracle.exact_value(bits[:cut]) + oracle.exact_value(bits[cut:])


GRID = [0.0, -0.0, 1.0, -1.0, 0.75, -3.0, math.ldexp(1.0, -1074), -math.ldexp(1.0, -1074),
        math.ldexp(1.0, -1022), math.ldexp(1.0 - 2.0 ** -52, -1022), math.ldexp(1.0, -53),
        math.ldexp(1.0, 1023), -math.ldexp(1.0, 1023), 1.7976931348623157e308, 1.0 + 2.0 ** -52]


def test_brute_force_grid():
    """Every sequence of length <= 3 from the grid against Fraction / float(Fraction)."""
    for n in range(1, 4):
        for combo in itertools.product(GRID, repeat=n):
            bits = np.array(combo, dtype=np.float64).view(np.uint64)
            S = sum(Fraction(v) for v in combo)
            r = oracle.exact_sum(bits)
            if S != 0:
                try:
                    want = float(S)
                except OverflowError:
                    want = math.inf if S > 0 else -math.inf
                assert r == fpref.from_float(want, F64), combo
                for mode in (RTZ, RUP, RDOWN):
                    fpref.check_rounding(S, oracle.exact_sum(bits, F64, F64, mode), F64, mode)
                for out in (F32, BF16):
                    fpref.check_rounding(S, oracle.exact_sum(bits, F64, out, RNE), out, RNE)
            else:
                signs = [math.copysign(1.0, v) < 0 for v in combo]
                zeros = all(v == 0 for v in combo)
                if zeros and all(signs):
                    assert r == 1 << 63
                else:
                    assert r == 0
                    rd = oracle.exact_sum(bits, F64, F64, RDOWN)
                    assert rd == (0 if zeros and not any(signs) else 1 << 63)


def test_segmented_oracle_against_fsum():
    rng = np.random.default_rng(12)
    lengths = np.array([0, 1, 5, 0, 300, 2, 1000], dtype=np.int64)
    off = W.csr_offsets(lengths)
    x = rng.uniform(-1, 1, int(off[-1]))
    res = oracle.exact_sum_segmented(x.view(np.uint64), off)
    for s in range(len(lengths)):
        seg = x[off[s]:off[s + 1]]
        assert int(res[s]) == fpref.from_float(math.fsum(seg.tolist()), F64)


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.exact_sum(np.zeros(3, dtype=np.uint64), F64, F64, 9)
    with pytest.raises(ValueError):
        oracle.exact_sum_segmented(np.zeros(3, dtype=np.uint64), np.array([0, 2, 1]))
