"""Exact sums of arrays sharded across processes (one GPU per rank).

The paper's MapReduce algorithm (Section 6.1) lets every reducer build a
superaccumulator of its share of the input and ends with one post-process
that adds the reducers' accumulators and rounds the total once.  Across
devices the same structure needs exactly one exchange:

1. every rank adds its shard into a zeroed device accumulator with the
   library's own kernel (``exactsum_acc_add``: the single-array reduction,
   with the grid's partials added into the caller's accumulator and the
   digits regularised so that |digit| <= 2^32);
2. the ranks add their accumulators word by word -- an integer SUM
   all-reduce of ``EXACTSUM_ACC_WORDS`` int64 words (640 bytes).  This is
   the carry-free superaccumulator addition of Section 2 (Lemma 1) with the
   carries deferred: regularised digits stay below 2^33 in magnitude after
   adding up to 2^30 of them, and the counter words (NaN / +Inf / -Inf seen,
   non-zero seen, element count) merge by the same addition;
3. every rank rounds the merged accumulator once on its device
   (``exactsum_acc_round``), so all ranks hold the same correctly rounded sum.

The exchange goes through whatever process group the caller set up: NCCL
moves the device tensor directly; any other backend (gloo on CPU) gets a
host copy of the 640 bytes and the merged words are copied back.  No rank
ever waits on another rank's kernel.
"""
from __future__ import annotations

from . import (ACC_WORDS, RNE, acc_add, acc_round, dtype_code, new_accumulator)


def allreduce_accumulator(acc, group=None):
    """In-place SUM all-reduce of an int64 accumulator tensor across ranks.

    A CUDA tensor is reduced in place when the group's backend is NCCL;
    otherwise (gloo) the words travel through a host copy.  Returns ``acc``.
    """
    import torch
    import torch.distributed as dist

    if acc.dtype != torch.int64 or acc.numel() != ACC_WORDS:
        raise TypeError(f"an accumulator is {ACC_WORDS} int64 words")
    backend = dist.get_backend(group)
    if acc.is_cuda and backend != "nccl":
        host = acc.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        acc.copy_(host)
    else:
        dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc


def sharded_accumulator(x_local, group=None, stream=None):
    """Steps 1-2: the merged accumulator of every rank's shard.

    ``x_local`` is this rank's contiguous CUDA tensor (float64 / float32 /
    bfloat16, or their raw bits); every rank must pass the same format.
    Returns the merged int64 accumulator on this rank's device.
    """
    import torch

    acc = new_accumulator(x_local.device)
    acc_add(acc, x_local, stream=stream)
    # the exchange must see the finished accumulator
    (stream or torch.cuda.current_stream(x_local.device)).synchronize()
    return allreduce_accumulator(acc, group=group)


def sharded_exact_sum(x_local, out_dtype=None, mode=RNE, group=None, stream=None):
    """The correctly rounded exact sum of the concatenation of every rank's
    shard (steps 1-3).  Returns a one-element tensor of the output format on
    this rank's device; every rank gets the same bits."""
    in_dtype = dtype_code(x_local)
    acc = sharded_accumulator(x_local, group=group, stream=stream)
    return acc_round(acc, in_dtype, in_dtype if out_dtype is None else out_dtype, mode, stream=stream)
