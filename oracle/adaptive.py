"""Oracle of the condition-number-sensitive summation (Section 4) over sparse
and r-truncated superaccumulators (Section 2, end), in plain Python.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Pure-Python loops:
meant for small inputs (up to some thousands of elements).

The steps, in the paper's order:

1. Each input element x_i becomes a sparse superaccumulator: its exact value
   in units of the format's smallest subnormal, written in radix R = 2^32,
   every component carrying the element's sign (|y_j| < R), only non-zero
   ("active") indices stored.  (The paper's radix is tied to the float
   mantissa; these are the integer digits its Section 2 also allows.)
2. A bottom-up summation tree of depth O(log n) over the leaves in input
   order: adjacent pairs are added level by level, an odd node moves up
   unchanged.
3. Each pairwise addition merges the active indices, adds corresponding
   components, and regularises them in one carry-free step (Lemma 1:
   P_i = y_i + z_i, carry c_i in {-1, 0, 1} chosen from P_i alone, here the
   balanced choice floor((P_i + R/2) / R); w_i = P_i - c_i R + c_{i-1}), and
   then keeps only the r most significant active components (the
   r-truncated sparse superaccumulator); the dropped components are counted.
4. The root's value is rounded once, y.
5. Stopping condition.  Every dropped component y_j satisfies |y_j| < R, so
   it is smaller than 2^(32(j+1)) units, and the total truncated mass is at
   most B = (components dropped) * 2^(32 (j_max + 1)) units.
     rule="rounded" (the reading the GPU path follows): stop when S - B and
       S + B round to y, S the root's exact value; then the exact sum, which
       lies within B of S, rounds to y as well.
     rule="paper_sound": stop when y (+) B = y (-) B = y, the paper's test
       ((+) a correctly rounded addition) with the bound B; y is then a
       faithful rounding of the exact sum.
     rule="paper": the paper's test as printed, with n * eps_min in place of
       B, eps_min the weight of the root's least significant kept
       component.  The paper argues that nothing truncated can reach that
       weight; with cancellation higher up the tree a partial sum can drop a
       component at or above it (the components above it cancel later), and
       the test can then accept a result that is not faithful (the tests
       keep such an input).  The GPU path therefore uses the bound B.
   If the test fails, r <- r^2 and the tree is summed again; once r reaches
   the number of digits the format can occupy nothing can be truncated and
   the exact sum is taken (one more pass).

Non-finite inputs and signed zeros are outside the paper; they follow the
exact oracle's rules (a NaN or an infinity decides the result whatever is
truncated).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .oracle import BF16, F32, F64, RDOWN, RNE, RUP, exact_sum, round_value

RADIX_BITS = 32
R = 1 << RADIX_BITS
_FMT = {  # exponent bits, fraction bits, unit exponent, digits the exact sum can occupy
    F64: (11, 52, -1074, 67),
    F32: (8, 23, -149, 10),
    BF16: (8, 7, -133, 9),
}
_WIDTH = {F64: 64, F32: 32, BF16: 16}


def element_value(bits: int, dt: int):
    """Exact value of one finite element in units, or None for NaN/Inf."""
    eb, fb, _, _ = _FMT[dt]
    w = _WIDTH[dt]
    s = (bits >> (w - 1)) & 1
    E = (bits >> fb) & ((1 << eb) - 1)
    F = bits & ((1 << fb) - 1)
    if E == (1 << eb) - 1:
        return None
    m = F if E == 0 else F + (1 << fb)
    p = max(E, 1) - 1
    v = m << p
    return -v if s else v


def leaf(value: int) -> dict:
    """Step 1: the sparse superaccumulator of one element's value."""
    sign = -1 if value < 0 else 1
    mag = abs(value)
    comps = {}
    i = 0
    while mag:
        d = mag & (R - 1)
        if d:
            comps[i] = sign * d
        mag >>= RADIX_BITS
        i += 1
    return comps


def merge(y: dict, z: dict) -> dict:
    """Step 3: add two regularised sparse superaccumulators (Lemma 1)."""
    P = dict(y)
    for i, v in z.items():
        P[i] = P.get(i, 0) + v
    carry_in = {}
    w = {}
    for i, p in P.items():
        c = (p + R // 2) // R  # balanced carry, in {-1, 0, 1} since |p| < 2R
        if p - c * R:
            w[i] = p - c * R
        if c:
            carry_in[i + 1] = c
    for i, c in carry_in.items():
        v = w.get(i, 0) + c
        if v:
            w[i] = v
        else:
            w.pop(i, None)
    return w


def truncate(y: dict, r: int, stats: dict) -> dict:
    """Step 3: keep the r most significant active components."""
    if len(y) <= r:
        return y
    keep = sorted(y, reverse=True)[:r]
    out = {i: y[i] for i in keep}
    for i in y:
        if i not in out:
            stats["dropped"] += 1
            stats["maxdrop"] = max(stats["maxdrop"], i)
    return out


def tree_sum(values: list, r: int, stats: dict) -> dict:
    """Step 2: bottom-up pairwise tree over the leaves, truncating each sum."""
    level = [leaf(v) for v in values]
    if not level:
        return {}
    while len(level) > 1:
        nxt = [truncate(merge(level[k], level[k + 1]), r, stats) for k in range(0, len(level) - 1, 2)]
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


def value_of(y: dict) -> int:
    return sum(v << (RADIX_BITS * i) for i, v in y.items())


def adaptive_sum(bits, in_dtype: int = F64, out_dtype: int = F64, mode: int = RNE,
                 rule: str = "rounded"):
    """Returns (result bits, passes, last r (0 for the exact pass))."""
    bits = np.asarray(bits)
    eb, fb, unit_exp, digits = _FMT[in_dtype]
    n = len(bits)
    values = [element_value(int(b), in_dtype) for b in bits]
    if n == 0 or any(v is None for v in values):
        return exact_sum(bits, in_dtype, out_dtype, mode, 1), 1, 0
    passes = 0
    r = 2
    while r < digits:
        passes += 1
        stats = {"dropped": 0, "maxdrop": -1}
        root = tree_sum(values, r, stats)
        S = value_of(root)
        if S == 0 and stats["dropped"] == 0:
            # an exact zero: the signed-zero rules decide
            return exact_sum(bits, in_dtype, out_dtype, mode, 1), passes, r
        y = round_value(S, unit_exp, out_dtype, mode)
        if stats["dropped"] == 0:
            return y, passes, r
        if rule == "rounded":
            B = stats["dropped"] << (RADIX_BITS * (stats["maxdrop"] + 1))
            if round_value(S - B, unit_exp, out_dtype, mode) == y and \
                    round_value(S + B, unit_exp, out_dtype, mode) == y:
                return y, passes, r
        else:
            if rule == "paper":
                lowest = min(root) if root else 0
                neps = n << (RADIX_BITS * lowest)
            else:
                neps = stats["dropped"] << (RADIX_BITS * (stats["maxdrop"] + 1))
            yv = float_units(y, out_dtype, unit_exp)
            if yv is not None and round_value(yv + neps, unit_exp, out_dtype, mode) == y and \
                    round_value(yv - neps, unit_exp, out_dtype, mode) == y:
                return y, passes, r
        r = r * r
    return exact_sum(bits, in_dtype, out_dtype, mode, 1), passes + 1, 0


def float_units(ybits: int, out_dtype: int, unit_exp: int):
    """A finite result's value in units of 2^unit_exp (None if it is not a
    finite multiple of that unit)."""
    eb, fb, _, _ = _FMT[out_dtype]
    w = _WIDTH[out_dtype]
    s = (ybits >> (w - 1)) & 1
    E = (ybits >> fb) & ((1 << eb) - 1)
    F = ybits & ((1 << fb) - 1)
    if E == (1 << eb) - 1:
        return None
    m = F if E == 0 else F + (1 << fb)
    bias = (1 << (eb - 1)) - 1
    val = Fraction(m) * Fraction(2) ** (max(E, 1) - bias - fb) / Fraction(2) ** unit_exp
    if val.denominator != 1:
        return None
    return -int(val) if s else int(val)


def is_faithful(ybits: int, bits, in_dtype: int, out_dtype: int) -> bool:
    """True when y is the exact sum or one of its two neighbours in the
    output format (finite results only)."""
    unit_exp = _FMT[in_dtype][2]
    S = sum(element_value(int(b), in_dtype) for b in bits)
    lo = round_value(S, unit_exp, out_dtype, RDOWN)
    hi = round_value(S, unit_exp, out_dtype, RUP)
    return ybits in (lo, hi)
