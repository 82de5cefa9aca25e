"""GPU parity of the single-array exact sum against the CPU oracle.

Bit-exact comparison (the method is exact; there is no tolerance): every
result of the CUDA path must equal the oracle's bit pattern.  Sizes span
many CTA tiles with ragged tails; pointers are also offset so that the
unaligned head path runs.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1605_05436_gb300 import workloads as W
from tests import gpu_util as G
from tests.test_oracle_pins import CLOSED, encode_inputs, expected_matches

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_05436_gb300 as es  # noqa: E402

DEV = "cuda:0"
MODES = (es.RNE, es.RTZ, es.RUP, es.RDOWN)


def gpu_sum(bits, i, o, m, offset=0):
    x = G.to_device(bits, i, DEV, offset)
    r = es.exact_sum(x, o, m)
    torch.cuda.synchronize()
    return G.result_bits(r, o)[0]


@pytest.mark.parametrize("case", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms_gpu(case):
    name, i, o, m, inputs, expected, why = case
    x = encode_inputs(inputs, i)
    r = gpu_sum(x, i, o, m)
    assert expected_matches(expected, r, o), f"{name}: got {r:#x} ({why})"
    assert r == oracle.exact_sum(x, i, o, m)


SIZES = [0, 1, 2, 3, 5, 8, 17, 31, 32, 33, 100, 767, 768, 769, 1000, 4097, 12345, 65536 + 3,
         (1 << 20) + 17, 3 * (1 << 20) + 5]


def make(dist, n, seed, dt):
    if dt == es.F64:
        if dist == "uniform":
            return W.uniform_f64(n, seed)
        if dist == "cancel":
            r = min(n, 64) if (n - min(n, 64)) % 2 == 0 else min(n, 63)
            return W.cancelling_f64(n, seed, residue=r)
        rng = np.random.default_rng(seed)
        return W._random_f64_bits(rng, n, -1022, 1023)
    if dt == es.F32:
        return W.wide_f32(n, seed) if dist != "uniform" else W.uniform_f32(n, seed)
    return W.wide_bf16(n, seed)


@pytest.mark.parametrize("dt", [es.F64, es.F32, es.BF16])
@pytest.mark.parametrize("dist", ["uniform", "cancel", "wide"])
def test_random_sizes(dt, dist):
    rng = np.random.default_rng(1000 * dt + len(dist))
    for n in SIZES:
        bits = make(dist, n, int(rng.integers(1 << 31)), dt)
        for o in (es.F64, es.F32, es.BF16):
            m = int(rng.integers(4))
            assert gpu_sum(bits, dt, o, m) == oracle.exact_sum(bits, dt, o, m, threads=8), (n, o, m)


@pytest.mark.parametrize("dt", [es.F64, es.F32, es.BF16])
def test_unaligned_heads_and_tails(dt):
    rng = np.random.default_rng(77 + dt)
    for off in range(1, 8):
        for n in (1, 2, 7, 9, 1023, 100_001):
            bits = make("wide", n, int(rng.integers(1 << 31)), dt)
            for m in MODES:
                assert gpu_sum(bits, dt, dt, m, offset=off) == oracle.exact_sum(bits, dt, dt, m, 4)


def test_specials_anywhere():
    """NaN / infinities placed at the head, middle and tail, alone and together."""
    rng = np.random.default_rng(5)
    n = 300_001
    base = W.uniform_f64(n, 9)
    specials = {"nan": 0x7FF8000000000001, "pinf": 0x7FF0000000000000, "ninf": 0xFFF0000000000000}
    for combo in (["nan"], ["pinf"], ["ninf"], ["pinf", "ninf"], ["pinf", "pinf"]):
        for where in (0, n // 2, n - 1, int(rng.integers(n))):
            bits = base.copy()
            for k, s in enumerate(combo):
                bits[(where + 7919 * k) % n] = specials[s]
            for o in (es.F64, es.F32, es.BF16):
                assert gpu_sum(bits, es.F64, o, es.RNE) == oracle.exact_sum(bits, es.F64, o, es.RNE, 8)


def test_signed_zero_rules():
    for n in (1, 5, 1000, 200_003):
        for pattern in ("negzero", "poszero", "mixed", "cancel", "subnormal_cancel"):
            if pattern == "negzero":
                bits = np.full(n, 1 << 63, dtype=np.uint64)
            elif pattern == "poszero":
                bits = np.zeros(n, dtype=np.uint64)
            elif pattern == "mixed":
                bits = np.where(np.arange(n) % 3 == 0, np.uint64(1 << 63), np.uint64(0)).astype(np.uint64)
            elif pattern == "cancel":
                v = W.uniform_f64(n // 2 + 1, n)
                bits = np.concatenate([v, v ^ np.uint64(1 << 63)])
            else:
                v = np.arange(1, n // 2 + 2, dtype=np.uint64)  # subnormals
                bits = np.concatenate([v, v ^ np.uint64(1 << 63)])
            for m in MODES:
                assert gpu_sum(bits, es.F64, es.F64, m) == oracle.exact_sum(bits, es.F64, es.F64, m, 4), (n, pattern, m)


def _constant_device(bits_value: int, n: int, dt: int):
    """n copies of one bit pattern, filled on the device (no host copy)."""
    signed = G.NP_SIGNED[dt](np.array([bits_value], dtype=G.NP_UNSIGNED[dt]).view(G.NP_SIGNED[dt])[0])
    return torch.full((n,), int(signed), dtype=G.torch_bits_dtype(dt), device=DEV)


@pytest.mark.parametrize("dt,n,E", [(es.F64, (1 << 27) + 3, 1024), (es.F32, (1 << 28) + 5, 8),
                                    (es.F32, (1 << 28) + 5, 32), (es.F32, (1 << 28) + 5, 254),
                                    (es.BF16, (1 << 34) + 7, 8), (es.BF16, (1 << 34) + 7, 15),
                                    (es.BF16, (1 << 30) + 7, 254)])
def test_regularisation_bound(dt, n, E):
    """Adversarial inputs at the deferred-carry headroom: every element adds
    the largest possible value to one digit (mantissa all ones at the
    largest in-digit offset), all positive, all negative, and then with
    alternating signs.  n is large enough that each thread regularises
    mid-stream.  The exact sums are closed forms (n * x, -n * x and x),
    rounded by the oracle.  For FP64 the largest offset is p = E - 1 with
    p mod 32 = 31; for FP32 both p mod 32 = 31 (E = 32: the radix-2^32
    columns, where each addition adds just under 2^55 to one 64-bit digit)
    and p mod 8 = 7 (E = 8), and the largest finite FP32 (E = 254, whose
    carries reach the top digit); for BF16 both the integer
    digits' worst case (p mod 8 = 7, E = 8) and the FP32 digits' worst case
    (E mod 8 = 7, E = 15: each addition adds 255 units of 2^-7 to one FP32
    digit, the most an addition can) are run, and the largest finite BF16
    (E = 254, the top FP32 digit, whose carries reach the top int32 digit)."""
    if dt == es.F64:
        v, unit, m = (E << 52) | ((1 << 52) - 1), -1074, (1 << 53) - 1   # p = 32*31 + 31
    elif dt == es.F32:
        v, unit, m = (E << 23) | 0x7FFFFF, -149, (1 << 24) - 1            # mantissa all ones
    else:
        v, unit, m = (E << 7) | 0x7F, -133, (1 << 8) - 1
    p = E - 1
    sign = 1 << (8 * es.ITEMSIZE[dt] - 1)
    x = _constant_device(v, n, dt)
    for o in (dt, es.F64):
        r = es.exact_sum(x, o, es.RNE)
        torch.cuda.synchronize()
        assert G.result_bits(r, o)[0] == oracle.round_value(n * (m << p), unit, o, es.RNE), o
    neg = _constant_device(v | sign, 1, dt)
    x.fill_(neg[0])
    for o in (dt, es.F64):
        r = es.exact_sum(x, o, es.RNE)
        torch.cuda.synchronize()
        assert G.result_bits(r, o)[0] == oracle.round_value(-n * (m << p), unit, o, es.RNE), o
    x[0::2] = _constant_device(v, 1, dt)[0]  # alternate signs: n is odd, so the sum is x itself
    r = es.exact_sum(x, dt, es.RNE)
    torch.cuda.synchronize()
    assert G.result_bits(r, dt)[0] == v
    del x


def test_extreme_magnitudes():
    """Sums that overflow and come back, max-exponent and min-subnormal mixes."""
    n = 100_000
    rng = np.random.default_rng(3)
    big = np.uint64(0x7FEFFFFFFFFFFFFF)
    bits = np.where(rng.random(n) < 0.5, big, big | np.uint64(1 << 63)).astype(np.uint64)
    bits[::97] = 1  # min subnormal
    for m in MODES:
        assert gpu_sum(bits, es.F64, es.F64, m) == oracle.exact_sum(bits, es.F64, es.F64, m, 8)
    bits = np.full(n, big, dtype=np.uint64)
    for m in MODES:
        for o in (es.F64, es.F32):
            assert gpu_sum(bits, es.F64, o, m) == oracle.exact_sum(bits, es.F64, o, m, 8)


def test_accumulator_chunks_and_merge():
    """Exactness of the carry-free accumulator: chunked adds, and two
    accumulators merged by plain integer addition, round to the whole sum."""
    bits = W.cancelling_f64((1 << 20) + 64, seed=4, residue=64)
    x = G.to_device(bits, es.F64, DEV)
    acc = es.new_accumulator(DEV)
    cuts = [0, 1, 1000, 333_333, 700_001, len(bits)]
    for a, b in zip(cuts[:-1], cuts[1:]):
        es.acc_add(acc, x[a:b])
    acc2 = es.new_accumulator(DEV)
    es.acc_add(acc2, x[:500_000])
    acc3 = es.new_accumulator(DEV)
    es.acc_add(acc3, x[500_000:])
    merged = acc2 + acc3
    for m in MODES:
        want = oracle.exact_sum(bits, es.F64, es.F64, m, 8)
        assert G.result_bits(es.acc_round(acc, es.F64, es.F64, m), es.F64)[0] == want
        assert G.result_bits(es.acc_round(merged, es.F64, es.F64, m), es.F64)[0] == want
    assert int(acc[77].item()) == len(bits)  # element count word


def test_sum_host_matches():
    for dt, bits in ((es.F64, W.cancelling_f64((1 << 23) + 1024, seed=8)),
                     (es.F32, W.wide_f32((1 << 22) + 3, seed=8)),
                     (es.BF16, W.wide_bf16((1 << 24) + 5, seed=8))):
        h = torch.from_numpy(bits.view(G.NP_SIGNED[dt])).pin_memory()
        for o in (dt, es.F64):
            got = es.exact_sum_host(h, o, es.RNE)
            assert got == oracle.exact_sum(bits, dt, o, es.RNE, 8)


def test_config1_full():
    """Single FP64 array, n = 2^20, uniform [-1, 1), seed 0, RNE."""
    bits = W.uniform_f64(1 << 20, 0)
    r = gpu_sum(bits, es.F64, es.F64, es.RNE)
    assert r == oracle.exact_sum(bits, threads=8)
    assert r == np.array([math.fsum(bits.view(np.float64).tolist())]).view(np.uint64)[0]


def test_config2_full():
    """Single FP64 array, n = 2^28 (2 GiB): +/- pairs over exponents
    [-1000, 1000] and 1024 uniform residues, shuffled; launched exactly as the
    benchmark launches it."""
    n = 1 << 28
    bits = W.cancelling_f64(n, seed=0)
    x = G.to_device(bits, es.F64, DEV)
    for m in MODES:
        r = es.exact_sum(x, es.F64, m)
        torch.cuda.synchronize()
        assert G.result_bits(r, es.F64)[0] == oracle.exact_sum(bits, es.F64, es.F64, m, threads=16)
    res = W.cancelling_residue(n, seed=0)
    want = np.array([math.fsum(res.view(np.float64).tolist())]).view(np.uint64)[0]
    r = es.exact_sum(x)
    assert G.result_bits(r, es.F64)[0] == want


def test_config3_full():
    """FP32 n = 2^29 (1% subnormals) and BF16 n = 2^30, rounded to the input
    format and to FP64."""
    b32 = W.wide_f32(1 << 29, seed=0)
    x = G.to_device(b32, es.F32, DEV)
    for o in (es.F32, es.F64):
        r = es.exact_sum(x, o, es.RNE)
        torch.cuda.synchronize()
        assert G.result_bits(r, o)[0] == oracle.exact_sum(b32, es.F32, o, es.RNE, threads=16)
    del x, b32
    b16 = W.wide_bf16(1 << 30, seed=0)
    x = G.to_device(b16, es.BF16, DEV)
    for o in (es.BF16, es.F64):
        r = es.exact_sum(x, o, es.RNE)
        torch.cuda.synchronize()
        assert G.result_bits(r, o)[0] == oracle.exact_sum(b16, es.BF16, o, es.RNE, threads=16)


def test_back_to_back_launches():
    """Consecutive FP64 sums on one stream may overlap on the device: the next
    launch starts streaming while the one before it merges and rounds, and
    waits for it only before it touches the handle's partials, ticket and
    result (programmatic dependent launch).  Sixteen different arrays (large
    enough for the launches to overlap) are summed back to back with no
    synchronisation in between, then eight of them are added back to back
    into one accumulator; every result must equal the oracle's."""
    arrays = []
    for k in range(16):
        n = (1 << 24) + 1001 * k
        arrays.append(W.cancelling_f64(n, seed=100 + k) if k % 2 == 0 else W.uniform_f64(n, seed=100 + k))
    xs = [G.to_device(b, es.F64, DEV, k % 3) for k, b in enumerate(arrays)]
    torch.cuda.synchronize()
    outs = [es.exact_sum(x, es.F64, es.RNE) for x in xs]
    torch.cuda.synchronize()
    for k, (b, r) in enumerate(zip(arrays, outs)):
        assert G.result_bits(r, es.F64)[0] == oracle.exact_sum(b, es.F64, es.F64, es.RNE, threads=8), k
    acc = es.new_accumulator(DEV)
    for x in xs[:8]:
        es.acc_add(acc, x)
    r = es.acc_round(acc, es.F64, es.F64, es.RNE)
    torch.cuda.synchronize()
    want = oracle.exact_sum(np.concatenate(arrays[:8]), es.F64, es.F64, es.RNE, threads=8)
    assert G.result_bits(r, es.F64)[0] == want
    del xs


def test_invalid_arguments():
    h = es.handle_for(0)
    x = torch.zeros(16, dtype=torch.float64, device=DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(es.ExactSumError) as ei:
        es.exactsum_sum(h, x.data_ptr(), 16, 7, es.F64, es.RNE, out.data_ptr(), s)
    assert ei.value.status == es.EINVAL
    with pytest.raises(es.ExactSumError):
        es.exactsum_sum(h, x.data_ptr(), -1, es.F64, es.F64, es.RNE, out.data_ptr(), s)
    with pytest.raises(es.ExactSumError):
        es.exactsum_sum(h, x.data_ptr(), 16, es.F64, es.F64, 9, out.data_ptr(), s)
    with pytest.raises(es.ExactSumError):
        es.exactsum_sum(h, x.data_ptr() + 4, 8, es.F64, es.F64, es.RNE, out.data_ptr(), s)
    with pytest.raises(es.ExactSumError):
        es.exactsum_sum(h, None, 5, es.F64, es.F64, es.RNE, out.data_ptr(), s)
    with pytest.raises(es.ExactSumError):
        es.exactsum_sum(h, x.data_ptr(), 5, es.F64, es.F64, es.RNE, None, s)
    # the handle is still usable after rejected calls
    x[:] = 1.0
    es.exactsum_sum(h, x.data_ptr(), 16, es.F64, es.F64, es.RNE, out.data_ptr(), s)
    torch.cuda.synchronize()
    assert out.item() == 16.0


NARROW_SPECIALS = {es.F32: {"nan": 0x7FC00001, "pinf": 0x7F800000, "ninf": 0xFF800000, "negzero": 0x80000000},
                   es.BF16: {"nan": 0x7FC1, "pinf": 0x7F80, "ninf": 0xFF80, "negzero": 0x8000}}


@pytest.mark.parametrize("dt", [es.F32, es.BF16])
def test_narrow_specials_anywhere(dt):
    """FP32/BF16 arrays long enough for the vector path (whose kernels decode
    two elements at once and keep the exponent maximum packed in 16-bit
    halves): NaN / infinities at even and odd positions (both halves of a
    decoded pair), alone and together."""
    rng = np.random.default_rng(31 + dt)
    n = 300_001
    base = W.uniform_f32(n, 9) if dt == es.F32 else W.wide_bf16(n, 9)
    sp = NARROW_SPECIALS[dt]
    for combo in (["nan"], ["pinf"], ["ninf"], ["pinf", "ninf"], ["ninf", "ninf"]):
        for where in (0, 1, n // 2, n // 2 + 1, n - 1, int(rng.integers(n))):
            bits = base.copy()
            for k, s in enumerate(combo):
                bits[(where + 7919 * k) % n] = sp[s]
            for o in (es.F64, dt):
                assert gpu_sum(bits, dt, o, es.RNE) == oracle.exact_sum(bits, dt, o, es.RNE, 8), (combo, where, o)


@pytest.mark.parametrize("dt", [es.F32, es.BF16])
def test_narrow_signed_zero_rules(dt):
    """All-zero FP32/BF16 arrays (every exponent maximum 0) take the exact
    classification: -0 only, +0 only, mixed, and cancelling subnormals."""
    neg = NARROW_SPECIALS[dt]["negzero"]
    ut = G.NP_UNSIGNED[dt]
    for n in (9, 1000, 200_003):
        for pattern in ("negzero", "poszero", "mixed", "subnormal_cancel"):
            if pattern == "negzero":
                bits = np.full(n, neg, dtype=ut)
            elif pattern == "poszero":
                bits = np.zeros(n, dtype=ut)
            elif pattern == "mixed":
                bits = np.where(np.arange(n) % 3 == 0, ut(neg), ut(0)).astype(ut)
            else:
                v = (np.arange(1, n // 2 + 2) % 100 + 1).astype(ut)  # subnormals
                bits = np.concatenate([v, v ^ ut(neg)])
            for m in MODES:
                assert gpu_sum(bits, dt, dt, m) == oracle.exact_sum(bits, dt, dt, m, 4), (n, pattern, m)
