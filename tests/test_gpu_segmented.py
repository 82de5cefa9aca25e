"""GPU parity of the batched (segmented) exact sum against the CPU oracle.

Bit-exact: every segment's result equals the oracle's.  Cases cover empty
segments, tile boundaries, unaligned segment starts, a non-zero first offset,
invalid offsets (NaN plus a device status bit), graph replay, the autotuner,
and the 65,536-segment Anderson-style workload (1/16 scale, and full size
on the benchmark's reducer, every segment checked)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1605_05436_gb300 import workloads as W
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_05436_gb300 as es  # noqa: E402

DEV = "cuda:0"


def run_segmented(bits, off, i, o, m):
    x = G.to_device(bits, i, DEV)
    d_off = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).to(DEV)
    r = es.segmented_sum(x, d_off, o, m)
    torch.cuda.synchronize()
    return np.array(G.result_bits(r, o), dtype=np.uint64)


def make_bits(dt, n, seed):
    if dt == es.F64:
        return W.cancelling_f64(n + (n % 2), seed, residue=0)[:n] if n > 1 else W.uniform_f64(n, seed)
    if dt == es.F32:
        return W.wide_f32(n, seed)
    return W.wide_bf16(n, seed)


EDGE_LENGTHS = [0, 1, 2, 3, 7, 8, 9, 31, 32, 33, 0, 0, 1000, 8191, 8192, 8193, 32767, 32768, 32769,
                65535, 65536, 65537, 131072 + 5, 0, 300_001, 1]


@pytest.mark.parametrize("dt", [es.F64, es.F32, es.BF16])
def test_edge_lengths(dt):
    lengths = np.array(EDGE_LENGTHS, dtype=np.int64)
    off = W.csr_offsets(lengths) + 3  # a non-zero first offset; unaligned starts
    bits = make_bits(dt, int(off[-1]) + 5, 11 + dt)
    for o in (dt, es.F64):
        for m in (es.RNE, es.RDOWN):
            got = run_segmented(bits, off, dt, o, m)
            want = oracle.exact_sum_segmented(bits, off, dt, o, m, threads=4)
            assert np.array_equal(got, want.astype(np.uint64)), (o, m)


def test_random_segments_all_modes():
    rng = np.random.default_rng(21)
    lengths = W.segment_lengths(700, seed=3, log2_max=17)
    lengths[rng.random(700) < 0.1] = 0
    off = W.csr_offsets(lengths)
    bits = W.segmented_f64(lengths, seed=4)
    for m in (es.RNE, es.RTZ, es.RUP, es.RDOWN):
        got = run_segmented(bits, off, es.F64, es.F64, m)
        want = oracle.exact_sum_segmented(bits, off, es.F64, es.F64, m, threads=8)
        assert np.array_equal(got, want.astype(np.uint64)), m


def test_segments_with_specials_and_zeros():
    lengths = np.array([5, 70_000, 3, 40_000, 2, 1, 100_000], dtype=np.int64)
    off = W.csr_offsets(lengths)
    bits = W.uniform_f64(int(off[-1]), 2)
    bits[off[0] + 1] = 0x7FF8000000000000  # NaN in segment 0
    bits[off[1] + 60_000] = 0x7FF0000000000000  # +Inf in a multi-tile segment
    bits[off[3] + 1] = 0xFFF0000000000000
    bits[off[3] + 39_000] = 0x7FF0000000000000  # +Inf and -Inf: NaN
    bits[off[4]:off[5]] = np.uint64(1 << 63)  # all -0
    bits[off[5]:off[6]] = 0  # +0
    bits[off[6]:off[7]] = np.concatenate([bits[off[6]:off[6] + 50_000],
                                          bits[off[6]:off[6] + 50_000] ^ np.uint64(1 << 63)])
    for m in (es.RNE, es.RDOWN):
        got = run_segmented(bits, off, es.F64, es.F64, m)
        want = oracle.exact_sum_segmented(bits, off, es.F64, es.F64, m, threads=4)
        assert np.array_equal(got, want.astype(np.uint64)), m


def test_bad_offsets_flagged():
    h = es.handle_for(0)
    es.exactsum_device_status(h)  # clear
    bits = W.uniform_f64(1000, 1)
    off = np.array([0, 100, 50, 1000], dtype=np.int64)  # segment 1 is negative
    got = run_segmented(bits, off, es.F64, es.F64, es.RNE)
    assert (int(got[1]) & 0x7FF0000000000000) == 0x7FF0000000000000 and int(got[1]) & 0xFFFFFFFFFFFFF
    assert int(got[0]) == oracle.exact_sum(bits[0:100])
    assert es.exactsum_device_status(h) & es.STATUS_BAD_OFFSETS
    assert es.exactsum_device_status(h) == 0  # cleared by the read


def test_matches_one_launch_per_segment_and_graph_replay():
    lengths = W.segment_lengths(500, seed=8, log2_max=16)
    off = W.csr_offsets(lengths)
    bits = W.segmented_f64(lengths, seed=9)
    x = G.to_device(bits, es.F64, DEV)
    d_off = torch.from_numpy(off).to(DEV)
    a = es.segmented_sum(x, d_off)
    b = es.segmented_sum(x, d_off)  # replays the cached graph
    c = es.sum_each(x, torch.from_numpy(off))
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))
    assert torch.equal(a.view(torch.int64), c.view(torch.int64))
    want = oracle.exact_sum_segmented(bits, off, threads=8)
    assert np.array_equal(np.array(G.result_bits(a, es.F64), dtype=np.uint64), want.astype(np.uint64))


def test_stream_capture_by_caller():
    """The caller may capture the segmented call into its own CUDA graph."""
    lengths = W.segment_lengths(300, seed=12, log2_max=15)
    off = W.csr_offsets(lengths)
    bits = W.segmented_f64(lengths, seed=13)
    x = G.to_device(bits, es.F64, DEV)
    d_off = torch.from_numpy(off).to(DEV)
    out = torch.empty(len(lengths), dtype=torch.float64, device=DEV)
    es.segmented_sum(x, d_off, out=out)  # grows the workspace outside capture
    torch.cuda.synchronize()
    out.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        es.segmented_sum(x, d_off, out=out)
    g.replay()
    torch.cuda.synchronize()
    want = oracle.exact_sum_segmented(bits, off, threads=8)
    assert np.array_equal(np.array(G.result_bits(out, es.F64), dtype=np.uint64), want.astype(np.uint64))


def test_autotune_and_tuning_file(tmp_path):
    lengths = W.segment_lengths(2048, seed=5, log2_max=16)
    off = W.csr_offsets(lengths)
    bits = W.segmented_f64(lengths, seed=6)
    x = G.to_device(bits, es.F64, DEV)
    d_off = torch.from_numpy(off).to(DEV)
    scratch = torch.empty(len(lengths), dtype=torch.float64, device=DEV)
    h = es.handle_for(0)
    s = torch.cuda.current_stream().cuda_stream
    warps, kind, tile, ms = es.exactsum_segmented_autotune(h, x.data_ptr(), d_off.data_ptr(), len(lengths),
                                                           es.F64, scratch.data_ptr(), s)
    assert warps in (8, 12, 16, 24, 32) and kind in (0, 1, 2) and tile > 0 and ms > 0
    p = str(tmp_path / "tuning.json")
    es.exactsum_tuning_save(h, p)
    text = open(p).read()
    assert '"warps": %d' % warps in text and '"tile": %d' % tile in text and '"kind": %d' % kind in text
    es.exactsum_tuning_load(h, p)
    got = es.segmented_sum(x, d_off)
    torch.cuda.synchronize()
    want = oracle.exact_sum_segmented(bits, off, threads=8)
    assert np.array_equal(np.array(G.result_bits(got, es.F64), dtype=np.uint64), want.astype(np.uint64))


@pytest.fixture(scope="module")
def anderson_full():
    lengths = W.segment_lengths(65536, seed=0)
    x = W.segmented_f64_device(lengths, seed=0, device=DEV)
    off = W.csr_offsets(lengths)
    return lengths, off, x


def test_anderson_sixteenth_scale():
    """4,096 segments of the 65,536-segment recipe, every segment checked."""
    lengths = W.segment_lengths(4096, seed=1)
    off = W.csr_offsets(lengths)
    x = W.segmented_f64_device(lengths, seed=1, device=DEV)
    d_off = torch.from_numpy(off).to(DEV)
    got = es.segmented_sum(x, d_off)
    torch.cuda.synchronize()
    bits = x.cpu().numpy().view(np.uint64)
    want = oracle.exact_sum_segmented(bits, off, threads=16)
    assert np.array_equal(np.array(G.result_bits(got, es.F64), dtype=np.uint64), want.astype(np.uint64))


def test_anderson_full_every_segment(anderson_full, tmp_path):
    """65,536 segments (about 5e9 elements, 40 GB) on the reducer the
    benchmark's autotuner picks for this workload (windowed, 24 warps,
    131,072-element tiles), launched as the benchmark launches it; the oracle
    checks every segment, and the handle's default reducer must agree."""
    import bench
    lengths, off, x = anderson_full
    d_off = torch.from_numpy(off).to(DEV)
    h = es.handle_for(0)
    S = len(lengths)
    try:
        _force_reducer(h, tmp_path, es.F64, S, 2, 131072)
        got = es.segmented_sum(x, d_off)
        torch.cuda.synchronize()
    finally:
        _restore_default(h, tmp_path, es.F64, S)
    got_bits = np.array(G.result_bits(got, es.F64), dtype=np.uint64)
    assert bench.oracle_check_segments(torch, x, off, got_bits) == []
    default = es.segmented_sum(x, d_off)
    torch.cuda.synchronize()
    assert np.array_equal(np.array(G.result_bits(default, es.F64), dtype=np.uint64), got_bits)
    assert es.exactsum_device_status(h) == 0


REDUCERS = {1: "tma", 2: "window"}


def _force_reducer(h, tmp_path, dt, S, kind, tile):
    lg = int(np.ceil(np.log2(S)))
    # the warps field must name the shape the library is built with
    warps = {1: 8 if dt == es.F64 else 12, 2: 24 if dt == es.F64 else 32}[kind]
    p = tmp_path / f"force_{dt}_{kind}_{tile}.json"
    p.write_text('{"segmented": [{"in_dtype": %d, "log2_segments": %d, "warps": %d, "kind": %d, '
                 '"tile": %d, "ms": -1}]}' % (dt, lg, warps, kind, tile))
    es.exactsum_tuning_load(h, str(p))


def _restore_default(h, tmp_path, dt, S):
    lg = int(np.ceil(np.log2(S)))
    p = tmp_path / f"reg_{dt}.json"
    p.write_text('{"segmented": [{"in_dtype": %d, "log2_segments": %d, "warps": 8, "kind": 0, "tile": %d}]}'
                 % (dt, lg, (256 << 10) // es.ITEMSIZE[dt]))
    es.exactsum_tuning_load(h, str(p))


@pytest.mark.parametrize("kind", [1, 2], ids=lambda k: REDUCERS[k])
@pytest.mark.parametrize("dt", [es.F64, es.F32, es.BF16])
def test_reducer_forms_forced(tmp_path, dt, kind):
    """The TMA-ring and windowed reducers (chosen through a tuning file) give
    the oracle's bits on edge lengths, with small and large tiles."""
    h = es.handle_for(0)
    lengths = np.array(EDGE_LENGTHS * 3, dtype=np.int64)
    off = W.csr_offsets(lengths) + 1
    bits = make_bits(dt, int(off[-1]) + 3, 40 + dt)
    S = len(lengths)
    try:
        for tile in (4096, 65536):
            _force_reducer(h, tmp_path, dt, S, kind, tile)
            for o, m in ((dt, es.RNE), (es.F64, es.RUP)):
                got = run_segmented(bits, off, dt, o, m)
                want = oracle.exact_sum_segmented(bits, off, dt, o, m, threads=8)
                assert np.array_equal(got, want.astype(np.uint64)), (tile, o, m)
    finally:
        _restore_default(h, tmp_path, dt, S)
    assert es.exactsum_device_status(h) & 4 == 0  # no wait timed out


@pytest.mark.parametrize("dt", [es.F64, es.F32, es.BF16])
def test_window_reducer_overflow_path(tmp_path, dt):
    """Segments whose exponents spread far beyond any window: nearly every
    element takes the windowed reducer's exact overflow path (and, for FP64,
    forces many overflow regularisations), and Anderson-style segments that
    stay inside the window.  Both must match the oracle."""
    h = es.handle_for(0)
    lengths = np.array([131072, 3, 200_000, 70_000, 1, 0, 50_000], dtype=np.int64)
    off = W.csr_offsets(lengths)
    n = int(off[-1])
    if dt == es.F64:
        wide = W.cancelling_f64(n + (n % 2), seed=77, residue=0, emin=-1000, emax=1000)[:n]
        narrow = W.segmented_f64(lengths, seed=78)
        cases = (wide, narrow)
    elif dt == es.F32:
        cases = (W.wide_f32(n, seed=79), W.uniform_f32(n, seed=80))
    else:
        cases = (W.wide_bf16(n, seed=81),)
    S = len(lengths)
    try:
        _force_reducer(h, tmp_path, dt, S, 2, 131072)
        for bits in cases:
            for m in (es.RNE, es.RDOWN):
                got = run_segmented(bits, off, dt, es.F64, m)
                want = oracle.exact_sum_segmented(bits, off, dt, es.F64, m, threads=8)
                assert np.array_equal(got, want.astype(np.uint64)), m
    finally:
        _restore_default(h, tmp_path, dt, S)
