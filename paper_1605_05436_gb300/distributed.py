"""Multi-device merge of exact partial sums.

An accumulator (``EXACTSUM_ACC_WORDS`` int64 words, see ``include/exactsum.h``)
holds regularised radix-2^32 digits plus counters.  Two accumulators of the
same input format merge by adding them word by word -- the carry-free
superaccumulator addition of Section 2 (Lemma 1) with deferred carries -- so
a sharded exact sum needs exactly one exchange: an integer SUM all-reduce of
640 bytes per device, followed by one rounding (``exactsum_acc_round``).
"""
from __future__ import annotations


def allreduce_accumulator(acc, group=None):
    """In-place SUM all-reduce of an int64 accumulator tensor across ranks
    (NCCL for CUDA tensors, gloo for CPU tensors).  Digits regularised by
    ``exactsum_acc_add`` satisfy |d| <= 2^32, so up to 2^30 ranks merge
    without overflow."""
    import torch
    import torch.distributed as dist

    if acc.dtype != torch.int64:
        raise TypeError("accumulators are int64 tensors")
    dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc
