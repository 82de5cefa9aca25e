"""Sharded exact sums through the library's own accumulators (world size 2).

Two processes share cuda:0 and a gloo process group.  Each one adds its own
shard into a device accumulator with the library's kernel
(``exactsum_acc_add``), the two accumulators are merged by one integer SUM
all-reduce (through a host copy, since gloo reduces CPU tensors), and each
rank rounds the merged accumulator on the GPU (``exactsum_acc_round``).
Both ranks must hold the same bits, equal to the CPU oracle's exact sum of
the concatenated input: the post-process of Section 6.1 on top of the
superaccumulator addition of Section 2 (Lemma 1).

No kernel of one rank waits on the other rank: the only exchange is the
gloo all-reduce on the host, between kernel launches.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1605_05436_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import torch.multiprocessing as mp  # noqa: E402

F64, F32, BF16 = 0, 1, 2
RNE, RTZ, RUP, RDOWN = 0, 1, 2, 3
NP_SIGNED = {F64: np.int64, F32: np.int32, BF16: np.int16}
NP_UNSIGNED = {F64: np.uint64, F32: np.uint32, BF16: np.uint16}
TORCH_BITS = {F64: "int64", F32: "int32", BF16: "int16"}


def _cases():
    """(name, in_dtype, out_dtype, mode, shard0 bits, shard1 bits)."""
    bits = W.cancelling_f64((1 << 20) + 1024, seed=31)
    cases = [("cancelling", F64, F64, RNE, bits[:400_001], bits[400_001:]),
             ("cancelling-rdown", F64, F64, RDOWN, bits[:7], bits[7:])]
    nan = W.uniform_f64(70_000, seed=32)
    nan_shard = nan[35_000:].copy()
    nan_shard[123] = 0x7FF8000000000000
    cases.append(("nan-on-rank1", F64, F64, RNE, nan[:35_000], nan_shard))
    negz = np.full(5000, 1 << 63, dtype=np.uint64)
    cases.append(("all-minus-zero", F64, F64, RNE, negz[:2000], negz[2000:]))
    cases.append(("minus-zero-and-plus-zero", F64, F64, RNE, negz[:2000], np.zeros(10, np.uint64)))
    f32 = W.wide_f32(300_000, seed=33)
    cases.append(("wide-f32-to-f64", F32, F64, RUP, f32[:100_000], f32[100_000:]))
    bf = W.wide_bf16(200_003, seed=34)
    cases.append(("wide-bf16", BF16, BF16, RNE, bf[:150_000], bf[150_000:]))
    u = W.uniform_f64(9_999, seed=35)
    cases.append(("empty-shard", F64, F64, RTZ, u[:0], u))
    return cases


def _worker(rank, port, q):
    import torch.distributed as dist

    import paper_1605_05436_gb300 as es
    from paper_1605_05436_gb300.distributed import sharded_accumulator, sharded_exact_sum

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        out = {}
        for name, i, o, m, s0, s1 in _cases():
            shard = np.ascontiguousarray((s0, s1)[rank]).view(NP_SIGNED[i])
            x = torch.from_numpy(shard.copy()).to(dev)
            r = sharded_exact_sum(x, out_dtype=o, mode=m)
            rb = int(r.view(getattr(torch, TORCH_BITS[o])).cpu().numpy().view(NP_UNSIGNED[o])[0])
            acc = sharded_accumulator(x)
            out[name] = (rb, int(acc[77].item()), int(acc[72].item()))
        q.put((rank, out))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_ranks_on_one_gpu_match_the_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = dict(q.get(timeout=600) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert got[0] == got[1]  # every rank rounds the same merged accumulator
    for name, i, o, m, s0, s1 in _cases():
        whole = np.concatenate([s0, s1])
        bits, count, nan_words = got[0][name]
        assert bits == oracle.exact_sum(whole, i, o, m, threads=8), name
        assert count == len(whole), name
        assert (nan_words > 0) == (name == "nan-on-rank1"), name
