"""The allocation-free segmented sum (exactsum_segmented_sum_noalloc).

It exists for callers that cannot allocate device memory (no handle, no
workspace): it keeps its scratch in a fixed array inside the library.  The
test calls it through the C ABI twice in a row -- the second time on other
data, so that whatever the first call left in the shared scratch would show
-- and checks each result against the regular entry point
(exactsum_segmented_sum) bit for bit, the tolerance every parity test here
uses, and against the CPU oracle.  It also checks the size limit.

This file is named so that pytest collects it last.
"""
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


def _case(seed, num_segments, dt):
    lengths = W.segment_lengths(num_segments, seed=seed, log2_max=17)
    lengths[::7] = 0  # empty segments too
    off = W.csr_offsets(lengths)
    if dt == es.F64:
        bits = W.segmented_f64(lengths, seed=seed + 1)
    elif dt == es.F32:
        bits = W.wide_f32(int(off[-1]), seed=seed + 1)
    else:
        bits = W.wide_bf16(int(off[-1]), seed=seed + 1)
    return bits, off


def _noalloc(x, d_off, num_segments, in_dt, out_dt, mode):
    out = es.result_tensor(out_dt, x.device, num_segments)
    es.exactsum_segmented_sum_noalloc(x.data_ptr(), d_off.data_ptr(), num_segments, in_dt, out_dt, mode,
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out


def test_noalloc_matches_regular_entry_point_twice():
    cases = [(_case(3, es.NOALLOC_MAX_SEGMENTS, es.F64), es.F64, es.F64, es.RNE),
             (_case(9, 1000, es.F32), es.F32, es.F64, es.RDOWN),
             (_case(5, 777, es.BF16), es.BF16, es.BF16, es.RNE),
             (_case(7, 500, es.F64), es.F64, es.F32, es.RTZ)]
    for (bits, off), in_dt, out_dt, mode in cases:
        x = G.to_device(bits, in_dt, DEV)
        d_off = torch.from_numpy(off).to(DEV)
        S = len(off) - 1
        regular = es.segmented_sum(x, d_off, out_dt, mode)
        got = _noalloc(x, d_off, S, in_dt, out_dt, mode)
        torch.cuda.synchronize()
        rb = np.array(G.result_bits(regular, out_dt), dtype=np.uint64)
        gb = np.array(G.result_bits(got, out_dt), dtype=np.uint64)
        assert np.array_equal(gb, rb)
        want = oracle.exact_sum_segmented(bits, off, in_dt, out_dt, mode, threads=8).astype(np.uint64)
        assert np.array_equal(gb, want)


def test_noalloc_bad_offsets_give_nan():
    """A segment whose end precedes its start gives a quiet NaN (no status is
    reported on this path); the valid segments beside it are exact."""
    bits = W.uniform_f64(1000, 1)
    x = G.to_device(bits, es.F64, DEV)
    off = np.array([0, 100, 50, 1000], dtype=np.int64)
    d_off = torch.from_numpy(off).to(DEV)
    got = _noalloc(x, d_off, 3, es.F64, es.F64, es.RNE)
    torch.cuda.synchronize()
    gb = G.result_bits(got, es.F64)
    assert (gb[1] & 0x7FF0000000000000) == 0x7FF0000000000000 and gb[1] & 0xFFFFFFFFFFFFF
    assert gb[0] == oracle.exact_sum(bits[0:100])
    assert gb[2] == oracle.exact_sum(bits[50:1000])


def test_noalloc_rejects_too_many_segments():
    x = torch.zeros(16, dtype=torch.float64, device=DEV)
    S = es.NOALLOC_MAX_SEGMENTS + 1
    d_off = torch.zeros(S + 1, dtype=torch.int64, device=DEV)
    out = torch.zeros(S, dtype=torch.float64, device=DEV)
    with pytest.raises(es.ExactSumError) as ei:
        es.exactsum_segmented_sum_noalloc(x.data_ptr(), d_off.data_ptr(), S, es.F64, es.F64, es.RNE,
                                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == es.EINVAL
    assert "maximum" in str(ei.value)
