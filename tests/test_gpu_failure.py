"""Failure detection on the GPU without a fault.

Every wait inside the library's kernels is bounded.  A wait that is never
satisfied gives up after its polls, the handle's device status word reports
EXACTSUM_STATUS_TIMEOUT through exactsum_device_status, and the CUDA
context stays usable: the next exact sum on the same handle is bit-exact
against the CPU oracle and reports nothing.  The failure is made by an
mbarrier that nothing ever completes (exactsum_check_timeout), polled a
bounded number of times by one thread: no trap, assert, bad address or
endless loop is involved.
"""
from __future__ import annotations

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


def _sum_bits(h, bits, n):
    x = G.to_device(bits, es.F64, DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    es.exactsum_sum(h, x.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    return G.result_bits(out, es.F64)[0]


@pytest.mark.parametrize("polls", [1, 1 << 16])
def test_unsatisfied_wait_reports_timeout_and_the_context_survives(polls):
    h = es.exactsum_create(0)
    try:
        assert es.exactsum_device_status(h) == 0
        elapsed = torch.zeros(1, dtype=torch.int64, device=DEV)
        es.exactsum_check_timeout(h, polls, elapsed.data_ptr(), torch.cuda.current_stream().cuda_stream)
        status = es.exactsum_device_status(h)
        assert status & es.STATUS_TIMEOUT
        assert status & ~es.STATUS_TIMEOUT == 0
        assert int(elapsed.item()) > 0
        assert es.exactsum_device_status(h) == 0  # reading the word cleared it
        n = 4097
        bits = W.uniform_f64(n, seed=11)
        assert _sum_bits(h, bits, n) == oracle.exact_sum(bits, es.F64, es.F64, es.RNE)
        assert es.exactsum_device_status(h) == 0
    finally:
        es.exactsum_destroy(h)


def test_timeout_on_one_handle_leaves_another_clean():
    h1, h2 = es.exactsum_create(0), es.exactsum_create(0)
    try:
        es.exactsum_check_timeout(h1, 1 << 10, None, torch.cuda.current_stream().cuda_stream)
        assert es.exactsum_device_status(h2) == 0
        assert es.exactsum_device_status(h1) & es.STATUS_TIMEOUT
    finally:
        es.exactsum_destroy(h1)
        es.exactsum_destroy(h2)


def test_check_timeout_argument_errors():
    h = es.exactsum_create(0)
    try:
        buf = torch.zeros(2, dtype=torch.int64, device=DEV)
        with pytest.raises(es.ExactSumError) as ei:
            es.exactsum_check_timeout(h, 1, buf.data_ptr() + 4, torch.cuda.current_stream().cuda_stream)
        assert ei.value.status == es.EINVAL
        assert es.exactsum_device_status(h) == 0  # nothing was enqueued
    finally:
        es.exactsum_destroy(h)


def test_the_kernels_own_limit_gives_up_in_about_a_second():
    # polls = 0 runs the kernels' own wait function with its own limit
    h = es.exactsum_create(0)
    try:
        elapsed = torch.zeros(1, dtype=torch.int64, device=DEV)
        es.exactsum_check_timeout(h, 0, elapsed.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert es.exactsum_device_status(h) == es.STATUS_TIMEOUT
        seconds = int(elapsed.item()) * 1e-9
        assert 0.05 < seconds < 10.0, seconds
    finally:
        es.exactsum_destroy(h)
