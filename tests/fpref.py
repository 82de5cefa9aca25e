"""Exact-rational helpers for the tests (no code shared with the oracle or
the CUDA library).

Values are taken from numpy's own float64/float32 conversions (bfloat16 is
the upper half of a float32), turned into ``fractions.Fraction`` exactly, and
results are checked by bracketing with numpy's ``nextafter`` -- the IEEE
definition of each rounding mode, not a re-implementation of one.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

F64, F32, BF16 = 0, 1, 2
RNE, RTZ, RUP, RDOWN = 0, 1, 2, 3
NP_BITS = {F64: np.uint64, F32: np.uint32, BF16: np.uint16}
SIGN_BIT = {F64: 1 << 63, F32: 1 << 31, BF16: 1 << 15}


def to_float(bits: int, dtype: int) -> float:
    """Python float (exact) of a bit pattern; bf16 and f32 widen exactly."""
    if dtype == F64:
        return float(np.array([bits], dtype=np.uint64).view(np.float64)[0])
    if dtype == F32:
        return float(np.array([bits], dtype=np.uint32).view(np.float32)[0])
    return float(np.array([bits << 16], dtype=np.uint32).view(np.float32)[0])


def from_float(v: float, dtype: int) -> int:
    """Bit pattern of a float that is exactly representable in dtype."""
    if dtype == F64:
        return int(np.array([v], dtype=np.float64).view(np.uint64)[0])
    f = np.float32(v)
    assert float(f) == v or math.isnan(v), "not representable"
    b = int(np.array([f], dtype=np.float32).view(np.uint32)[0])
    if dtype == F32:
        return b
    assert b & 0xFFFF == 0 or math.isnan(v), "not representable in bf16"
    return b >> 16


def exact(bits_array, dtype: int) -> Fraction:
    """Exact rational sum of the finite elements."""
    total = Fraction(0)
    for b in np.asarray(bits_array).tolist():
        v = to_float(int(b), dtype)
        if math.isfinite(v):
            total += Fraction(v)
    return total


def next_up(bits: int, dtype: int) -> int:
    """Bit pattern of the next representable value toward +inf."""
    if dtype == F64:
        v = np.array([bits], dtype=np.uint64).view(np.float64)
        with np.errstate(over="ignore"):
            return int(np.nextafter(v, np.inf).view(np.uint64)[0])
    if dtype == F32:
        v = np.array([bits], dtype=np.uint32).view(np.float32)
        with np.errstate(over="ignore"):
            return int(np.nextafter(v, np.float32(np.inf)).view(np.uint32)[0])
    # bfloat16: step the 16-bit pattern (sign-magnitude ordering)
    if bits == 0x8000:
        return 0x0001
    return bits + 1 if not bits & 0x8000 else bits - 1


def next_down(bits: int, dtype: int) -> int:
    neg = bits ^ SIGN_BIT[dtype]
    return next_up(neg, dtype) ^ SIGN_BIT[dtype]


def is_nan(bits: int, dtype: int) -> bool:
    return math.isnan(to_float(bits, dtype))


def check_rounding(S: Fraction, r: int, dtype: int, mode: int) -> None:
    """Assert that bit pattern r is the correctly rounded value of the exact
    rational S in format dtype under mode (S != 0)."""
    v = to_float(r, dtype)
    assert not math.isnan(v)
    if math.isinf(v):
        # every finite value must be a worse answer: the largest finite value
        # of the same sign is rejected by the mode's rule
        mx_bits = next_down(r, dtype) if v > 0 else next_up(r, dtype)
        mx = Fraction(to_float(mx_bits, dtype))
        if mode == RNE:
            # the overflow threshold is max + half an ulp of max
            ulp = mx - Fraction(to_float(next_down(mx_bits, dtype) if v > 0
                                         else next_up(mx_bits, dtype), dtype))
            assert abs(S) >= abs(mx) + abs(ulp) / 2
        elif mode == RTZ:
            raise AssertionError("round toward zero never overflows to infinity")
        elif mode == RUP:
            assert v > 0 and S > mx
        else:
            assert v < 0 and S < mx
        return
    R = Fraction(v)
    up = to_float(next_up(r, dtype), dtype)
    dn = to_float(next_down(r, dtype), dtype)
    if mode == RDOWN:
        assert R <= S and (math.isinf(up) or S < Fraction(up))
    elif mode == RUP:
        assert R >= S and (math.isinf(dn) or S > Fraction(dn))
    elif mode == RTZ:
        if S > 0:
            assert R <= S and (math.isinf(up) or S < Fraction(up))
        else:
            assert R >= S and (math.isinf(dn) or S > Fraction(dn))
    else:
        err = abs(S - R)
        for nb in (up, dn):
            if math.isinf(nb):
                continue
            e2 = abs(S - Fraction(nb))
            assert err <= e2, (S, R, nb)
            if err == e2:  # a tie: the kept value has an even last bit
                assert r & 1 == 0
    # the sign of a non-zero result follows S (a zero result keeps S's sign)
    if v != 0:
        assert (v > 0) == (S > 0)
    else:
        assert (r & SIGN_BIT[dtype] != 0) == (S < 0)
