"""CPU oracle for the exact-summation path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The library under
``paper_1605_05436_gb300`` never imports it.
"""
from .oracle import (build, exact_sum, exact_sum_segmented, exact_value, round_value,
                     F64, F32, BF16, RNE, RTZ, RUP, RDOWN)
from .adaptive import adaptive_sum

__all__ = ["build", "exact_sum", "exact_sum_segmented", "exact_value", "round_value", "adaptive_sum",
           "F64", "F32", "BF16", "RNE", "RTZ", "RUP", "RDOWN"]
