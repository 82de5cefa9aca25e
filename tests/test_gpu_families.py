"""The paper's four dataset families (Section 6.3: all positive, mixed
signs, Anderson's mean-subtracted data, exact sum zero) over exponent ranges
delta from 10 to 2046: GPU results equal the oracle bit for bit, in every
rounding mode."""
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


@pytest.mark.parametrize("family", [1, 2, 3, 4])
@pytest.mark.parametrize("delta", [10, 100, 1000, 2046])
def test_family_delta(family, delta):
    n = (1 << 18) + 17
    bits = W.family_f64(family, n, delta, seed=family * 7 + delta)
    x = G.to_device(bits, es.F64, "cuda:0")
    for mode in (es.RNE, es.RTZ, es.RUP, es.RDOWN):
        r = es.exact_sum(x, es.F64, mode)
        torch.cuda.synchronize()
        assert G.result_bits(r, es.F64)[0] == oracle.exact_sum(bits, es.F64, es.F64, mode, threads=8), mode
    if family == 4:
        assert G.result_bits(es.exact_sum(x), es.F64)[0] == 0  # exact zero, +0
