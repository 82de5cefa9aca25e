"""Seeded synthetic inputs for the exact-summation path.

This module only draws numbers.  It holds none of the summation arithmetic
(no decoding into digits, no accumulation, no rounding), so both the CUDA
path and the CPU oracle can take their inputs from here without sharing any
of the method's code.

The paper's experiments (Section 6.3) use the four Zhu-Hayes dataset families
(all positive; mixed sign; Anderson's mean-subtracted data; sum exactly zero)
with an exponent-range parameter delta.  Their generator is not available, so
the functions below stand in for them with explicit recipes:

* ``uniform_f64``          mixed-sign uniform values (dataset 2).
* ``cancelling_f64``       +/- pairs with exponents over [-1000, 1000]
                           (delta ~ 2000) plus a small residue (dataset 4).
* ``wide_f32``/``wide_bf16`` every normal exponent plus subnormals.
* ``segmented_f64``        Anderson-style mean-subtracted segments (dataset 3)
                           with log-uniform segment lengths.
* ``serving_requests``     a Poisson request stream over a value pool.

All generators use numpy's PCG64 via ``default_rng(seed)``.  Floating-point
inputs are returned as unsigned-integer bit patterns (``uint64`` / ``uint32``
/ ``uint16``) so that every value, including subnormals, signed zeros,
infinities and NaN payloads, crosses every boundary untouched.
"""
from __future__ import annotations

import math

import numpy as np

F64, F32, BF16 = 0, 1, 2
DTYPE_NAMES = {F64: "f64", F32: "f32", BF16: "bf16"}
BITS_NP = {F64: np.uint64, F32: np.uint32, BF16: np.uint16}
ITEMSIZE = {F64: 8, F32: 4, BF16: 2}


def uniform_f64(n: int, seed: int = 0) -> np.ndarray:
    """n values uniform in [-1, 1) (float64), returned as uint64 bits."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n).view(np.uint64)


def uniform_f32(n: int, seed: int = 0) -> np.ndarray:
    """n float32 values uniform in [-1, 1), returned as uint32 bits."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n).astype(np.float32).view(np.uint32)


def _random_f64_bits(rng, count: int, emin: int, emax: int) -> np.ndarray:
    """Random-sign normal doubles: unbiased exponent uniform in [emin, emax],
    52-bit fraction uniform, hidden bit implied."""
    sign = rng.integers(0, 2, count, dtype=np.uint64)
    biased = rng.integers(emin + 1023, emax + 1023 + 1, count, dtype=np.uint64)
    frac = rng.integers(0, 1 << 52, count, dtype=np.uint64)
    return (sign << np.uint64(63)) | (biased << np.uint64(52)) | frac


def cancelling_f64(n: int, seed: int = 0, residue: int = 1024,
                   emin: int = -1000, emax: int = 1000) -> np.ndarray:
    """Ill-conditioned FP64 input of exactly n elements.

    (n - residue) / 2 random-sign values with exponent uniform over
    [emin, emax] and a uniform 52-bit fraction, their exact negations, and
    ``residue`` values uniform in [-1, 1); the whole array is shuffled.  The
    exact sum equals the exact sum of the residue values.  At n = 2^28 this
    is the 2 GiB delta ~ 2000 workload.
    """
    if residue > n or (n - residue) % 2:
        raise ValueError("n - residue must be even and non-negative")
    rng = np.random.default_rng(seed)
    half = (n - residue) // 2
    out = np.empty(n, dtype=np.uint64)
    out[:half] = _random_f64_bits(rng, half, emin, emax)
    out[half:2 * half] = out[:half] ^ np.uint64(1 << 63)
    out[2 * half:] = rng.uniform(-1.0, 1.0, residue).view(np.uint64)
    rng.shuffle(out)
    return out


def cancelling_residue(n: int, seed: int = 0, residue: int = 1024,
                       emin: int = -1000, emax: int = 1000) -> np.ndarray:
    """The residue values of ``cancelling_f64`` (same seed), as uint64 bits.

    Replays the generator's draws without building the pairs, so that a test
    can sum the 1024 residue values independently of the 2^28-element array.
    """
    rng = np.random.default_rng(seed)
    half = (n - residue) // 2
    _random_f64_bits(rng, half, emin, emax)
    return rng.uniform(-1.0, 1.0, residue).view(np.uint64)


def family_f64(family: int, n: int, delta: int, seed: int = 0) -> np.ndarray:
    """One of the four dataset families of the paper's experiments (Section
    6.3), with exponents spread over a range of width ``delta`` (centred on
    0, at most 2046 wide):

    1. all positive (condition number 1);
    2. mixed signs, uniform random;
    3. Anderson's ill-conditioned data: mixed signs, minus the float mean;
    4. exact sum zero: random values and their exact negations, shuffled.

    Values are random-sign (positive for family 1) doubles with unbiased
    exponent uniform in [-delta/2, delta/2] and a uniform 52-bit fraction.
    """
    if not 1 <= family <= 4:
        raise ValueError("family is 1..4")
    delta = max(0, min(int(delta), 2046))
    emin, emax = -(delta // 2), delta - delta // 2
    emin, emax = max(emin, -1022), min(emax, 1023)
    rng = np.random.default_rng(seed)
    if family == 4:
        half = n // 2
        out = np.empty(n, dtype=np.uint64)
        out[:half] = _random_f64_bits(rng, half, emin, emax)
        out[half:2 * half] = out[:half] ^ np.uint64(1 << 63)
        if n % 2:
            out[-1] = 0
        rng.shuffle(out)
        return out
    bits = _random_f64_bits(rng, n, emin, emax)
    if family == 1:
        bits &= np.uint64((1 << 63) - 1)
    if family == 3:
        x = bits.view(np.float64)
        with np.errstate(over="ignore", invalid="ignore"):
            mean = x.mean()
        if np.isfinite(mean):
            x = x - mean
        bits = x.view(np.uint64)
    return bits


def wide_f32(n: int, seed: int = 0, subnormal_frac: float = 0.01) -> np.ndarray:
    """FP32 bits: random sign; with probability 1 - subnormal_frac a normal with
    biased exponent uniform in [1, 254] and uniform 23-bit fraction, else a
    subnormal with fraction uniform in [1, 2^23)."""
    rng = np.random.default_rng(seed)
    sign = rng.integers(0, 2, n, dtype=np.uint32)
    biased = rng.integers(1, 255, n, dtype=np.uint32)
    frac = rng.integers(0, 1 << 23, n, dtype=np.uint32)
    sub = rng.random(n) < subnormal_frac
    biased[sub] = 0
    frac[sub] = rng.integers(1, 1 << 23, int(sub.sum()), dtype=np.uint32)
    return (sign << np.uint32(31)) | (biased << np.uint32(23)) | frac


def wide_bf16(n: int, seed: int = 0) -> np.ndarray:
    """BF16 bits: random sign, unbiased exponent uniform in [-126, 127]
    (biased 1..254), 7-bit fraction uniform."""
    rng = np.random.default_rng(seed)
    sign = rng.integers(0, 2, n, dtype=np.uint16)
    biased = rng.integers(1, 255, n, dtype=np.uint16)
    frac = rng.integers(0, 1 << 7, n, dtype=np.uint16)
    return (sign << np.uint16(15)) | (biased << np.uint16(7)) | frac


def segment_lengths(num_segments: int, seed: int = 0, log2_max: int = 20) -> np.ndarray:
    """Log-uniform segment lengths L = max(1, floor(2^(log2_max * U)))."""
    rng = np.random.default_rng(seed)
    u = rng.random(num_segments)
    return np.maximum(1, np.floor(np.exp2(log2_max * u))).astype(np.int64)


def csr_offsets(lengths: np.ndarray) -> np.ndarray:
    """int64 CSR offsets (S + 1 entries) for the given segment lengths."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def segmented_f64(lengths: np.ndarray, seed: int = 0, kmin: int = -200,
                  kmax: int = 200) -> np.ndarray:
    """Anderson-style segments: per segment k ~ U{kmin..kmax}, values
    N(0,1) * 2^k, then the segment's float64 mean is subtracted.
    Returned as uint64 bits, concatenated in segment order.  Intended for the
    host-side (small) variants; the full 40 GB case is drawn on the device
    by ``segmented_f64_device``."""
    rng = np.random.default_rng(seed)
    total = int(lengths.sum())
    out = np.empty(total, dtype=np.float64)
    pos = 0
    ks = rng.integers(kmin, kmax + 1, len(lengths))
    for L, k in zip(lengths.tolist(), ks.tolist()):
        v = rng.standard_normal(L) * math.ldexp(1.0, k)
        if L:
            v -= v.mean()
        out[pos:pos + L] = v
        pos += L
    return out.view(np.uint64)


def segmented_f64_device(lengths: np.ndarray, seed: int = 0, kmin: int = -200,
                         kmax: int = 200, device="cuda", batch_elems: int = 1 << 28):
    """Device-side draw of the same family as ``segmented_f64`` for sizes that
    do not fit a host-side generation budget (about 5e9 elements, 40 GB).

    Uses a seeded ``torch.Generator`` on the device.  Values differ from the
    numpy variant (different generator) but follow the same recipe.  Returns
    a float64 CUDA tensor.  Segments are generated in batches of consecutive
    segments holding at most ``batch_elems`` elements.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rng = np.random.default_rng(seed)
    ks = rng.integers(kmin, kmax + 1, len(lengths))
    total = int(lengths.sum())
    x = torch.empty(total, dtype=torch.float64, device=device)
    lens_t = torch.as_tensor(lengths, device=device)
    scale_t = torch.as_tensor(np.ldexp(1.0, ks), dtype=torch.float64, device=device)
    off = csr_offsets(lengths)
    s = 0
    S = len(lengths)
    while s < S:
        e = s
        while e < S and (off[e + 1] - off[s] <= batch_elems or e == s):
            e += 1
        lo, hi = int(off[s]), int(off[e])
        ids = torch.repeat_interleave(torch.arange(e - s, device=device, dtype=torch.int32),
                                      lens_t[s:e])
        v = torch.randn(hi - lo, generator=g, dtype=torch.float64, device=device)
        v.mul_(scale_t[s:e][ids])
        sums = torch.zeros(e - s, dtype=torch.float64, device=device)
        sums.index_add_(0, ids, v)
        mean = sums / lens_t[s:e].to(torch.float64)
        v.sub_(mean[ids])
        x[lo:hi] = v
        del ids, v
        s = e
    return x


def serving_requests(num_requests: int, seed: int = 0, mean_gap_us: float = 50.0,
                     log2_min: int = 10, log2_max: int = 26, p_f64: float = 0.8,
                     pool_log2: int = 26):
    """A Poisson request stream.

    Returns a dict of numpy arrays: ``arrival_us`` (cumulative exponential
    gaps), ``n`` (floor(2^(log2_min + (log2_max - log2_min) U))), ``dtype``
    (F64 with probability p_f64, else F32) and ``offset`` (a uniform window
    start into a 2^pool_log2-element value pool of that dtype).
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap_us, num_requests)
    arrival = np.cumsum(gaps) - gaps[0]
    u = rng.random(num_requests)
    n = np.floor(np.exp2(log2_min + (log2_max - log2_min) * u)).astype(np.int64)
    pool = 1 << pool_log2
    n = np.minimum(n, pool)
    dt = np.where(rng.random(num_requests) < p_f64, F64, F32).astype(np.int32)
    offset = (rng.random(num_requests) * (pool - n + 1)).astype(np.int64)
    return {"arrival_us": arrival, "n": n, "dtype": dt, "offset": offset}


def serving_pools(pool_log2: int = 26, seed: int = 0):
    """Value pools for the request stream: uniform [-1, 1) FP64 and FP32."""
    n = 1 << pool_log2
    return {F64: uniform_f64(n, seed), F32: uniform_f32(n, seed + 1)}
