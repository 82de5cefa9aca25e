"""GPU parity of the condition-number-sensitive sum (r-truncated passes,
r <- r^2, Section 4) against the oracle.

The stopping condition used on the GPU accepts a pass only when every
value within the truncation bound of the pass's sum rounds to the same
result, so the result is unique: the correctly rounded exact sum, compared
bit for bit with the exact oracle (and, on small inputs, with the
condition-number-sensitive oracle, whose summation tree differs).  The
number of passes depends on the tree and is checked against what the
inputs' structure fixes.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import adaptive as A
from paper_1605_05436_gb300 import workloads as W
from tests import gpu_util as G
from tests.test_oracle_pins import CLOSED, encode_inputs, expected_matches

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_05436_gb300 as es  # noqa: E402

DEV = "cuda:0"
MODES = (es.RNE, es.RTZ, es.RUP, es.RDOWN)


def gpu_adaptive(bits, i, o, m, offset=0):
    x = G.to_device(bits, i, DEV, offset)
    r, passes, last_r = es.adaptive_sum(x, o, m)
    return G.result_bits(r, o)[0], passes, last_r


@pytest.mark.parametrize("case", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(case):
    name, i, o, m, inputs, expected, why = case
    x = encode_inputs(inputs, i)
    r, _, _ = gpu_adaptive(x, i, o, m)
    assert expected_matches(expected, r, o), f"{name}: got {r:#x} ({why})"


@pytest.mark.parametrize("n", [1, 2, 3, 33, 769, 4097, 65536 + 3, (1 << 20) + 17])
@pytest.mark.parametrize("dist", ["uniform", "cancel", "wide"])
def test_f64_matches_oracle(dist, n):
    rng = np.random.default_rng(n)
    if dist == "uniform":
        bits = W.uniform_f64(n, seed=n)
    elif dist == "cancel":
        r = min(n, 64) if (n - min(n, 64)) % 2 == 0 else min(n, 63)
        bits = W.cancelling_f64(n, seed=n, residue=r)
    else:
        bits = W._random_f64_bits(rng, n, -1022, 1023)
    for m in MODES:
        for o in (es.F64, es.F32):
            y, passes, _ = gpu_adaptive(bits, es.F64, o, m, offset=n % 3)
            assert y == oracle.exact_sum(bits, es.F64, o, m, 8), (dist, n, m, o)
            assert 1 <= passes <= 4


@pytest.mark.parametrize("dt", [es.F32, es.BF16])
@pytest.mark.parametrize("n", [5, 1000, 123457, (1 << 22) + 9])
def test_narrow_matches_oracle(dt, n):
    bits = W.wide_f32(n, seed=n) if dt == es.F32 else W.wide_bf16(n, seed=n)
    for m in MODES:
        for o in (dt, es.F64):
            y, passes, _ = gpu_adaptive(bits, dt, o, m)
            assert y == oracle.exact_sum(bits, dt, o, m, 8)
            assert 1 <= passes <= 3


def test_small_inputs_agree_with_the_adaptive_oracle():
    for seed in range(4):
        for bits in (W.uniform_f64(1500, seed=seed), W.cancelling_f64(1524, seed=seed),
                     W.family_f64(2, 1500, 800, seed=seed)):
            assert gpu_adaptive(bits, es.F64, es.F64, es.RNE)[0] == A.adaptive_sum(bits)[0]


def test_passes_follow_the_structure():
    # small integers: one radix-2^32 part per element, within two digits
    ints = np.arange(1, 100001, dtype=np.float64).view(np.uint64)
    y, passes, last_r = gpu_adaptive(ints, es.F64, es.F64, es.RNE)
    assert y == oracle.exact_sum(ints) and (passes, last_r) == (1, 2)
    # the delta ~ 2000 cancelling workload: every truncated pass drops parts
    # of partial sums far above the result's last place -> the exact pass
    bits = W.cancelling_f64(1 << 20, seed=0)
    y, passes, last_r = gpu_adaptive(bits, es.F64, es.F64, es.RNE)
    assert y == oracle.exact_sum(bits, threads=8) and (passes, last_r) == (4, 0)
    # uniform [-1, 1): r = 2 keeps 64 bits below the running sums' top and
    # must fail; r = 4 keeps 128 and is enough
    bits = W.uniform_f64(1 << 22, seed=1)
    y, passes, last_r = gpu_adaptive(bits, es.F64, es.F64, es.RNE)
    assert y == oracle.exact_sum(bits, threads=8) and (passes, last_r) == (2, 4)


def test_specials_and_zeros():
    nan = np.array([1.0, math.nan, 2.0] * 1000, dtype=np.float64).view(np.uint64)
    assert gpu_adaptive(nan, es.F64, es.F64, es.RNE)[0] == oracle.exact_sum(nan)
    infs = np.array([math.inf, -math.inf, 3.0], dtype=np.float64).view(np.uint64)
    assert gpu_adaptive(infs, es.F64, es.F64, es.RNE)[0] == oracle.exact_sum(infs)
    negz = np.array([-0.0] * 777, dtype=np.float64).view(np.uint64)
    for m in MODES:
        assert gpu_adaptive(negz, es.F64, es.F64, m)[0] == oracle.exact_sum(negz, es.F64, es.F64, m)
    cancel = np.array([1e300, 1.0, -1e300, -1.0] * 500, dtype=np.float64).view(np.uint64)
    for m in MODES:
        assert gpu_adaptive(cancel, es.F64, es.F64, m)[0] == oracle.exact_sum(cancel, es.F64, es.F64, m)
    empty = np.zeros(0, dtype=np.uint64)
    assert gpu_adaptive(empty, es.F64, es.F64, es.RNE) == (0, 1, 0)


def test_full_size_cancelling_workload():
    """The 2^28-element delta ~ 2000 benchmark input: the adaptive path
    needs all four passes and returns the exact kernel's result."""
    n = 1 << 28
    x = torch.from_numpy(W.cancelling_f64(n, seed=0).view(np.int64)).to(DEV)
    r, passes, last_r = es.adaptive_sum(x)
    e = es.exact_sum(x)
    torch.cuda.synchronize()
    assert (passes, last_r) == (4, 0)
    assert G.result_bits(r, es.F64) == G.result_bits(e, es.F64)
