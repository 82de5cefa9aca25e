"""World-size-2 gloo test of the multi-device exchange: accumulators built
on separate ranks merge by one integer SUM all-reduce and round to the exact
sum of the whole input (the oracle's answer).  Runs on CPU."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ACC_WORDS, ACC_DIGITS = 80, 72
W_NAN, W_COUNT = 72, 77


def digits_of(value: int):
    """Regularised radix-2^32 digits of an exact integer (|d| <= 2^31)."""
    d = []
    for _ in range(ACC_DIGITS - 1):
        lo = value & 0xFFFFFFFF
        if lo >= 1 << 31:
            lo -= 1 << 32
        d.append(lo)
        value = (value - lo) >> 32
    d.append(value)
    return d


def value_of(words) -> int:
    return sum(int(w) << (32 * i) for i, w in enumerate(words[:ACC_DIGITS]))


def _worker(rank, world, port, shards, nan_rank, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1605_05436_gb300.distributed import allreduce_accumulator
    bits = shards[rank]
    acc = torch.zeros(ACC_WORDS, dtype=torch.int64)
    acc[:ACC_DIGITS] = torch.tensor(digits_of(oracle.exact_value(bits)), dtype=torch.int64)
    acc[W_COUNT] = len(bits)
    acc[W_NAN] = 1 if rank == nan_rank else 0
    allreduce_accumulator(acc)
    q.put((rank, acc.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("nan_rank", [-1, 1])
def test_two_rank_merge(nan_rank):
    import oracle
    from paper_1605_05436_gb300 import workloads as W
    bits = W.cancelling_f64((1 << 16) + 64, seed=5, residue=64)
    shards = [bits[:30_000].copy(), bits[30_000:].copy()]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, shards, nan_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1]  # every rank holds the merged accumulator
    merged = out[0]
    assert value_of(merged) == oracle.exact_value(bits)
    assert merged[W_COUNT] == len(bits)
    assert (merged[W_NAN] > 0) == (nan_rank >= 0)
    # the merged value rounds to the oracle's answer for the whole input
    assert oracle.round_value(value_of(merged), -1074) == oracle.exact_sum(bits, threads=2)
