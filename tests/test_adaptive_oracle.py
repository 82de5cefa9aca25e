"""Pins of the condition-number-sensitive oracle (Section 4 over sparse,
r-truncated superaccumulators, Section 2) against what the mathematics
fixes: plain integer addition, exact rationals, the faithfulness bracket,
the exact oracle's results, and iteration counts that follow from the
inputs' structure."""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import adaptive as A
from paper_1605_05436_gb300 import workloads as W

F64, F32, BF16 = oracle.F64, oracle.F32, oracle.BF16
MODES = (oracle.RNE, oracle.RTZ, oracle.RUP, oracle.RDOWN)


def f64_bits(xs):
    return np.asarray(xs, dtype=np.float64).view(np.uint64)


def random_sparse(rng, k, lo=0, hi=70):
    idx = rng.choice(np.arange(lo, hi), size=k, replace=False)
    return {int(i): int(rng.integers(-(1 << 32) + 1, 1 << 32)) for i in idx}


def test_leaf_is_the_value():
    rng = np.random.default_rng(0)
    for b in W.uniform_f64(200, seed=3).tolist() + W.cancelling_f64(1224, seed=4)[:200].tolist():
        v = A.element_value(int(b), F64)
        y = A.leaf(v)
        assert A.value_of(y) == v
        assert all(0 < abs(c) < A.R and (c > 0) == (v > 0) for c in y.values())
    del rng


def test_merge_is_integer_addition_and_regularises():
    """Lemma 1: the merged components are again in (-R, R) and the value is
    the plain integer sum."""
    rng = np.random.default_rng(1)
    for _ in range(500):
        y = random_sparse(rng, int(rng.integers(0, 12)))
        z = random_sparse(rng, int(rng.integers(0, 12)))
        w = A.merge(y, z)
        assert A.value_of(w) == A.value_of(y) + A.value_of(z)
        assert all(0 < abs(c) < A.R for c in w.values())
        # the balanced carry keeps components within R/2 + 1
        assert all(abs(c) <= A.R // 2 + 1 for c in w.values())


def test_truncate_keeps_the_most_significant_and_bounds_the_loss():
    rng = np.random.default_rng(2)
    for r in (1, 2, 4, 16):
        for _ in range(200):
            y = random_sparse(rng, int(rng.integers(0, 30)))
            st = {"dropped": 0, "maxdrop": -1}
            t = A.truncate(dict(y), r, st)
            assert len(t) == min(r, len(y))
            assert sorted(t) == sorted(y)[len(y) - len(t):]
            assert st["dropped"] == len(y) - len(t)
            loss = abs(A.value_of(y) - A.value_of(t))
            if st["dropped"]:
                assert loss < st["dropped"] << (32 * (st["maxdrop"] + 1))
            else:
                assert loss == 0


@pytest.mark.parametrize("family", ["uniform", "cancelling", "wide_range", "ints"])
def test_rounded_rule_gives_the_exact_oracle_result(family):
    rng = np.random.default_rng(7)
    for trial in range(4):
        n = int(rng.integers(1, 1500))
        if family == "uniform":
            bits = W.uniform_f64(n, seed=trial)
        elif family == "cancelling":
            bits = W.cancelling_f64(1024 + 2 * n, seed=trial)
        elif family == "wide_range":
            bits = W.family_f64(1, n, 1500, seed=trial)
        else:
            bits = f64_bits(rng.integers(-1000, 1000, n).astype(np.float64))
        for m in MODES:
            y, passes, _ = A.adaptive_sum(bits, F64, F64, m)
            assert y == oracle.exact_sum(bits, F64, F64, m, 2), (family, n, m)
            assert 1 <= passes <= 4
        # RNE pinned to Python's correctly rounded rational-to-float conversion
        exact = sum(Fraction(float(v)) for v in bits.view(np.float64))
        y, _, _ = A.adaptive_sum(bits)
        assert struct.unpack("<d", struct.pack("<Q", y))[0] == float(exact) or \
            (float(exact) == 0.0 and y in (0, 1 << 63))


@pytest.mark.parametrize("dt", [F32, BF16])
def test_narrow_formats(dt):
    for seed in range(3):
        bits = W.wide_f32(900, seed=seed) if dt == F32 else W.wide_bf16(900, seed=seed)
        for out in (dt, F64):
            for m in MODES:
                y, passes, _ = A.adaptive_sum(bits, dt, out, m)
                assert y == oracle.exact_sum(bits, dt, out, m, 2)
                assert 1 <= passes <= 3


def test_paper_test_with_the_sound_bound_is_faithful():
    """The paper's stopping test (y unchanged by adding or subtracting a
    bound of everything truncated) with the bound taken from the highest
    dropped component gives a faithful result: the exact sum or one of its
    neighbours in the output format."""
    for seed in range(6):
        for bits in (W.uniform_f64(700, seed=seed), W.cancelling_f64(1524, seed=seed),
                     W.family_f64(2, 700, 600, seed=seed)):
            y, _, _ = A.adaptive_sum(bits, rule="paper_sound")
            assert A.is_faithful(y, bits, F64, F64)


def test_printed_bound_fails_under_cancellation():
    """The bound as printed (n times the weight of the root's least
    significant kept component) misses components dropped at or above that
    weight lower in the tree.  On this ill-conditioned input (pairs with
    exponents over [-1000, 1000] and 500 residues) pass r = 16 keeps root
    digits 46..48 while a digit-48 component was dropped, and the printed
    test accepts a result that is not faithful; the sound bound does not."""
    bits = W.cancelling_f64(1524, seed=3)
    vals = [A.element_value(int(b), F64) for b in bits]
    st = {"dropped": 0, "maxdrop": -1}
    root = A.tree_sum(vals, 16, st)
    assert st["maxdrop"] >= min(root)
    y, passes, r = A.adaptive_sum(bits, rule="paper")
    assert (passes, r) == (3, 16) and not A.is_faithful(y, bits, F64, F64)
    assert A.adaptive_sum(bits, rule="paper_sound")[0] == oracle.exact_sum(bits)
    assert A.adaptive_sum(bits)[0] == oracle.exact_sum(bits)


def test_passes_follow_the_structure():
    # small integers: every element is one component at one index, partial
    # sums never hold more than two active components -> nothing truncated
    ints = f64_bits(np.arange(1, 2000, dtype=np.float64))
    assert A.adaptive_sum(ints)[1:] == (1, 2)
    # an ill-conditioned shuffle (pairs with exponents over [-1000, 1000]):
    # r = 2 must drop components of the big partial sums, far above the
    # result's last place, so more than one pass is needed
    y, passes, _ = A.adaptive_sum(W.cancelling_f64(3000, seed=2))
    assert passes > 1
    # the number of passes grows with the condition number
    rng = np.random.default_rng(5)
    base = rng.uniform(-1, 1, 256)
    last = 0
    for k in (0, 60, 400, 1000):
        big = rng.uniform(1, 2, 300) * 2.0 ** k
        xs = np.concatenate([base, big, -big])
        rng.shuffle(xs)
        p = A.adaptive_sum(xs.view(np.uint64))[1]
        assert p >= last
        last = p
    assert last > 2


def test_specials_and_empty():
    assert A.adaptive_sum(np.zeros(0, dtype=np.uint64)) == (0, 1, 0)
    nan = f64_bits([1.0, math.nan, 2.0])
    assert A.adaptive_sum(nan)[0] == oracle.exact_sum(nan)
    inf = f64_bits([math.inf, -5.0, 1e300])
    assert A.adaptive_sum(inf)[0] == 0x7FF0000000000000
    negz = f64_bits([-0.0, -0.0])
    assert A.adaptive_sum(negz)[0] == 1 << 63


def test_mutant_without_carries_is_caught(monkeypatch):
    """A merge that forgets the incoming carries (a plausible slip in
    Lemma 1) breaks the value identity."""
    def bad_merge(y, z):
        P = dict(y)
        for i, v in z.items():
            P[i] = P.get(i, 0) + v
        return {i: p - ((p + A.R // 2) // A.R) * A.R for i, p in P.items() if p - ((p + A.R // 2) // A.R) * A.R}
    monkeypatch.setattr(A, "merge", bad_merge)
    bits = W.uniform_f64(500, seed=1)
    assert A.adaptive_sum(bits)[0] != oracle.exact_sum(bits)
