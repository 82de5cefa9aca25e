"""The seeded input generators follow their stated recipes (CPU only)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1605_05436_gb300 import workloads as W


def test_cancelling_structure():
    n = (1 << 16) + 1024
    bits = W.cancelling_f64(n, seed=2)
    assert bits.dtype == np.uint64 and len(bits) == n
    res = W.cancelling_residue(n, seed=2)
    assert len(res) == 1024
    # every non-residue value appears with its exact negation
    rest = np.setdiff1d(bits, res)
    neg = rest ^ np.uint64(1 << 63)
    assert np.array_equal(np.sort(rest), np.sort(neg))
    # exponents of the pairs lie in [-1000, 1000]
    e = ((rest >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    assert e.min() >= -1000 and e.max() <= 1000 and e.max() - e.min() > 1900
    assert oracle.exact_value(bits) == oracle.exact_value(res)
    # shuffled: the pairs are not adjacent halves
    assert not np.array_equal(bits[: len(rest) // 2] ^ np.uint64(1 << 63), bits[len(rest) // 2: len(rest)])


def test_wide_f32_and_bf16():
    b = W.wide_f32(200_000, seed=1)
    e = (b >> np.uint32(23)) & np.uint32(0xFF)
    frac = b & np.uint32(0x7FFFFF)
    sub = e == 0
    assert 0.008 < sub.mean() < 0.012
    assert (frac[sub] > 0).all()
    assert e[~sub].min() == 1 and e[~sub].max() == 254
    h = W.wide_bf16(200_000, seed=1)
    e16 = (h >> np.uint16(7)) & np.uint16(0xFF)
    assert e16.min() == 1 and e16.max() == 254
    assert 0.45 < ((h >> np.uint16(15)) == 1).mean() < 0.55


def test_segment_lengths_log_uniform():
    L = W.segment_lengths(65536, seed=0)
    assert L.min() >= 1 and L.max() <= 1 << 20
    lg = np.log2(L)
    assert abs(lg.mean() - 10) < 0.2
    total = int(L.sum())
    assert 4.5e9 < total < 5.5e9  # about 4.96e9 elements expected
    off = W.csr_offsets(L)
    assert off[0] == 0 and off[-1] == total and (np.diff(off) == L).all()


def test_segmented_values_are_mean_subtracted():
    L = np.array([0, 1, 5, 1000], dtype=np.int64)
    bits = W.segmented_f64(L, seed=4)
    x = bits.view(np.float64)
    off = W.csr_offsets(L)
    for s in range(len(L)):
        seg = x[off[s]:off[s + 1]]
        if len(seg) > 1:
            assert abs(seg.mean()) <= 1e-12 * np.abs(seg).max()


def test_serving_requests_recipe():
    r = W.serving_requests(100_000, seed=0)
    gaps = np.diff(r["arrival_us"])
    assert 48 < gaps.mean() < 52
    assert r["n"].min() >= 1 << 10 and r["n"].max() <= 1 << 26
    assert 0.79 < (r["dtype"] == W.F64).mean() < 0.81
    assert (r["offset"] >= 0).all() and (r["offset"] + r["n"] <= 1 << 26).all()
    assert 5.5e6 < r["n"].mean() < 6.6e6  # about 6.05e6 elements per request
