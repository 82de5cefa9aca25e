"""GPU tests of the serving engine (continuous batching of exact-sum
requests): every result equals the oracle's, a request gives the same bits
alone and inside a mix, admission honours the memory budget, host-memory
requests are staged, requests spanning many tiles or steps keep their
partial sums in their device slots, and every lane configuration (resident
express kernel, express steps, bulk launches) gives the oracle's bits."""
from __future__ import annotations

import time

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


def collect(server, expected_count, timeout_s=120):
    es.exactsum_server_drain(server, int(timeout_s * 1000))
    recs = []
    while len(recs) < expected_count:
        got = es.exactsum_server_poll(server)
        if not got:
            break
        recs.extend(got)
    return {r.id: r for r in recs}


@pytest.fixture(scope="module")
def pools():
    p64 = W.uniform_f64(1 << 22, seed=3)
    p32 = W.wide_f32(1 << 22, seed=4)
    p16 = W.wide_bf16(1 << 22, seed=5)
    return {es.F64: (p64, G.to_device(p64, es.F64, DEV)),
            es.F32: (p32, G.to_device(p32, es.F32, DEV)),
            es.BF16: (p16, G.to_device(p16, es.BF16, DEV))}


@pytest.mark.parametrize("max_steps,lanes", [(0, None), (0, (-1, 16, 0)), (3, (-1, 16, 0)), (3, (1 << 20, 16, 0))],
                         ids=["default-lanes", "steps-only", "steps-only-max3", "steps-and-bulk"])
def test_mixed_requests_match_oracle(pools, max_steps, lanes):
    """Mixed sizes, formats, outputs and modes: with the default lanes (a
    resident express kernel and the bulk lane), and with the express lane
    as continuous-batching steps (every request, or beside the bulk lane),
    where requests span several steps (chunk 2^16, or at most 3 steps)."""
    server = es.exactsum_server_create(0, 64, 1 << 30, 1 << 16, 1 << 12, max_steps)
    try:
        if lanes:
            es.exactsum_server_set_lanes(server, *lanes)
        rng = np.random.default_rng(1)
        sizes = [0, 1, 2, 3, 63, 64, 65, 4095, 4096, 4097, 65535, 65536, 65537, 300_001, 1 << 21]
        reqs = {}
        for k, n in enumerate(sizes * 2):
            dt = [es.F64, es.F32, es.BF16][k % 3]
            out = [dt, es.F64][k % 2]
            mode = k % 4
            bits, dx = pools[dt]
            off = int(rng.integers(0, len(bits) - n + 1))
            ptr = dx[off:].data_ptr() if n else 0
            rid = es.exactsum_server_submit(server, ptr, n, dt, out, mode, 0)
            reqs[rid] = (bits[off:off + n], dt, out, mode)
        recs = collect(server, len(reqs))
        assert len(recs) == len(reqs)
        for rid, (b, dt, out, mode) in reqs.items():
            r = recs[rid]
            assert r.status == es.OK
            mask = (1 << (8 * es.ITEMSIZE[out])) - 1
            assert (r.result_bits & mask) == oracle.exact_sum(b, dt, out, mode, threads=8), (len(b), dt, out, mode)
            assert r.submit_ns <= r.admit_ns <= r.done_ns
    finally:
        es.exactsum_server_destroy(server)


def test_alone_equals_in_the_mix(pools):
    """The same request, alone and among 300 concurrent ones, gives the same bits."""
    bits, dx = pools[es.F64]
    n, off = 3_000_017, 12345
    want = oracle.exact_sum(bits[off:off + n], threads=8)
    server = es.exactsum_server_create(0, 32, 1 << 28, 1 << 17, 1 << 13)
    try:
        rid = es.exactsum_server_submit(server, dx[off:].data_ptr(), n, es.F64, es.F64, es.RNE, 0)
        alone = collect(server, 1)[rid].result_bits
        rng = np.random.default_rng(7)
        ids = []
        target = None
        for k in range(300):
            if k == 150:
                target = es.exactsum_server_submit(server, dx[off:].data_ptr(), n, es.F64, es.F64, es.RNE, 0)
            m = int(rng.integers(1, 1 << 18))
            o = int(rng.integers(0, len(bits) - m))
            ids.append(es.exactsum_server_submit(server, dx[o:].data_ptr(), m, es.F64, es.F64, es.RNE, 0))
        recs = collect(server, 301)
        assert recs[target].result_bits == alone == want
        stats = es.exactsum_server_stats(server)
        assert stats["peak_active"] > 1  # it really was a mix
    finally:
        es.exactsum_server_destroy(server)


def test_memory_budget_limits_residency(pools):
    bits, dx = pools[es.F64]
    n = 100_000  # 800 KB per request
    budget = 3 * (n * 8 + 640)  # room for three resident requests
    server = es.exactsum_server_create(0, 64, budget, 1 << 14, 1 << 12)
    try:
        ids = {}
        for k in range(40):
            o = 1000 * k
            ids[es.exactsum_server_submit(server, dx[o:].data_ptr(), n, es.F64, es.F64, es.RNE, 0)] = o
        recs = collect(server, 40)
        assert es.exactsum_server_stats(server)["peak_active"] <= 3
        for rid, o in ids.items():
            assert recs[rid].result_bits == oracle.exact_sum(bits[o:o + n], threads=4)
        # a request larger than the whole budget still runs (alone)
        big = es.exactsum_server_submit(server, dx.data_ptr(), 1 << 20, es.F64, es.F64, es.RNE, 0)
        assert collect(server, 1)[big].result_bits == oracle.exact_sum(bits[:1 << 20], threads=8)
    finally:
        es.exactsum_server_destroy(server)


def test_host_memory_requests(pools):
    server = es.exactsum_server_create(0, 16, 1 << 30, 1 << 16, 1 << 12)
    try:
        keep = []
        reqs = {}
        for k, (dt, n) in enumerate([(es.F64, 1 << 20), (es.F32, 777_777), (es.BF16, 123_457), (es.F64, 5)]):
            bits = pools[dt][0][:n]
            h = torch.from_numpy(bits.view(G.NP_SIGNED[dt]).copy()).pin_memory()
            keep.append(h)
            reqs[es.exactsum_server_submit(server, h.data_ptr(), n, dt, es.F64, es.RNE, 1)] = (bits, dt)
        recs = collect(server, len(reqs))
        for rid, (bits, dt) in reqs.items():
            assert recs[rid].status == es.OK
            assert recs[rid].result_bits == oracle.exact_sum(bits, dt, es.F64, es.RNE, threads=8)
    finally:
        es.exactsum_server_destroy(server)


def test_specials_across_steps(pools):
    """A NaN or an infinity in a late chunk of a many-step request."""
    bits = pools[es.F64][0][:1 << 20].copy()
    cases = []
    for pos, val in ((900_000, 0x7FF8000000000000), (500_000, 0xFFF0000000000000)):
        b = bits.copy()
        b[pos] = val
        cases.append(b)
    b = bits.copy()
    b[10] = 0x7FF0000000000000
    b[1_000_000] = 0xFFF0000000000000
    cases.append(b)
    server = es.exactsum_server_create(0, 8, 1 << 30, 1 << 15, 1 << 12)
    try:
        devs = [G.to_device(b, es.F64, DEV) for b in cases]
        ids = [es.exactsum_server_submit(server, d.data_ptr(), len(b), es.F64, es.F64, es.RNE, 0)
               for d, b in zip(devs, cases)]
        recs = collect(server, len(ids))
        for rid, b in zip(ids, cases):
            assert recs[rid].result_bits == oracle.exact_sum(b, threads=4)
    finally:
        es.exactsum_server_destroy(server)


def test_poisson_stream_sample(pools):
    """A short Poisson stream at 20k requests/s over windows of the pools."""
    req = W.serving_requests(2000, seed=11, log2_max=20, pool_log2=22)
    server = es.exactsum_server_create(0, 128, 4 << 30, 1 << 20, 1 << 14)
    try:
        ids = {}
        t0 = time.perf_counter()
        for k in range(len(req["n"])):
            while (time.perf_counter() - t0) * 1e6 < req["arrival_us"][k]:
                pass
            dt = int(req["dtype"][k])
            n, o = int(req["n"][k]), int(req["offset"][k])
            dx = pools[dt][1]
            ids[es.exactsum_server_submit(server, dx[o:].data_ptr(), n, dt, dt, es.RNE, 0)] = (dt, n, o)
        recs = collect(server, len(ids))
        assert len(recs) == len(ids)
        rng = np.random.default_rng(0)
        for rid in rng.choice(list(ids), 100, replace=False).tolist():
            dt, n, o = ids[rid]
            mask = (1 << (8 * es.ITEMSIZE[dt])) - 1
            assert (recs[rid].result_bits & mask) == oracle.exact_sum(pools[dt][0][o:o + n], dt, dt, es.RNE, 4)
    finally:
        es.exactsum_server_destroy(server)


def test_invalid_requests():
    server = es.exactsum_server_create(0, 4, 1 << 20, 1 << 12, 1 << 12)
    try:
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_submit(server, 0, 10, es.F64, es.F64, es.RNE, 0)
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_submit(server, 8, 10, 5, es.F64, es.RNE, 0)
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_submit(server, 8, 10, es.F64, es.F64, 7, 0)
    finally:
        es.exactsum_server_destroy(server)
    with pytest.raises(es.ExactSumError):
        es.exactsum_server_create(0, 0, 1 << 20, 1 << 12, 1 << 12)
    with pytest.raises(es.ExactSumError):
        es.exactsum_server_create(0, 4, 1 << 20, 1000, 64)  # chunk not a multiple of the tile


@pytest.mark.parametrize("resident", [1, 0])
@pytest.mark.parametrize("express_max_bytes", [-1, 0, 1 << 18])
def test_lanes_match_oracle(pools, express_max_bytes, resident):
    """Every request through the express lane only (-1), the bulk lane only
    (0: every non-empty request is larger), and a split at 256 KiB, with
    the express lane as a resident kernel or as steps, with device- and
    host-memory inputs, every format, output and mode: each result equals
    the oracle's, and a request gives the same bits whichever lane it takes."""
    server = es.exactsum_server_create(0, 64, 1 << 30, 1 << 16, 1 << 12, 2)
    try:
        es.exactsum_server_set_lanes(server, express_max_bytes, 16, resident)
        rng = np.random.default_rng(5)
        sizes = [0, 1, 7, 4096, 32_769, 65_537, 300_001, 1 << 20, (1 << 21) + 3]
        reqs, keep = {}, []
        for k, n in enumerate(sizes * 3):
            dt = [es.F64, es.F32, es.BF16][k % 3]
            out = [dt, es.F64, es.F32][(k // 3) % 3]
            mode = (k * 7) % 4
            bits, dx = pools[dt]
            off = int(rng.integers(0, len(bits) - n + 1))
            if k % 5 == 4 and n:
                h = torch.from_numpy(bits[off:off + n].view(G.NP_SIGNED[dt]).copy()).pin_memory()
                keep.append(h)
                rid = es.exactsum_server_submit(server, h.data_ptr(), n, dt, out, mode, 1)
            else:
                rid = es.exactsum_server_submit(server, dx[off:].data_ptr() if n else 0, n, dt, out, mode, 0)
            reqs[rid] = (bits[off:off + n], dt, out, mode)
        recs = collect(server, len(reqs))
        assert len(recs) == len(reqs)
        for rid, (b, dt, out, mode) in reqs.items():
            r = recs[rid]
            assert r.status == es.OK
            assert r.result_bits < (1 << (8 * es.ITEMSIZE[out]))
            assert r.result_bits == oracle.exact_sum(b, dt, out, mode, threads=8), (len(b), dt, out, mode)
    finally:
        es.exactsum_server_destroy(server)


def test_lanes_are_set_before_the_first_request(pools):
    server = es.exactsum_server_create(0, 8, 1 << 30, 1 << 15, 1 << 12)
    try:
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_set_lanes(server, 1 << 20, 0)
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_set_lanes(server, 1 << 20, 100_000)
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_set_lanes(server, 1 << 20, 8, 2)
        es.exactsum_server_set_lanes(server, 1 << 20, 8)
        bits, dx = pools[es.F64]
        rid = es.exactsum_server_submit(server, dx.data_ptr(), 1000, es.F64, es.F64, es.RNE, 0)
        with pytest.raises(es.ExactSumError):
            es.exactsum_server_set_lanes(server, 1 << 22, 16)
        assert collect(server, 1)[rid].result_bits == oracle.exact_sum(bits[:1000], threads=2)
    finally:
        es.exactsum_server_destroy(server)


def test_resident_kernel_leaves_when_idle_and_comes_back(pools):
    """The resident express kernel leaves after 5 ms without requests; the
    next request launches it again.  Requests spaced 20 ms apart (so the
    kernel has left before each) and bursts in between are all exact, and
    the engine counts the relaunches."""
    bits, dx = pools[es.F64]
    server = es.exactsum_server_create(0, 32, 1 << 30, 1 << 16, 1 << 12)
    try:
        rng = np.random.default_rng(17)
        want = {}
        for round_ in range(4):
            time.sleep(0.02)
            for k in range(1 + 5 * round_):
                n = int(rng.integers(1, 1 << 18))
                o = int(rng.integers(0, len(bits) - n))
                want[es.exactsum_server_submit(server, dx[o:].data_ptr(), n, es.F64, es.F64, es.RNE, 0)] = (o, n)
            recs = collect(server, len(want))
            for rid, (o, n) in want.items():
                assert recs[rid].status == es.OK
                assert recs[rid].result_bits == oracle.exact_sum(bits[o:o + n], threads=2), (round_, rid)
            want.clear()
        assert es.exactsum_server_stats(server)["steps"] >= 4  # express-lane kernel launches
    finally:
        es.exactsum_server_destroy(server)


def test_concurrent_submitters(pools):
    """Four host threads submit at once (the submit call is thread-safe):
    every request, from either lane, gives the oracle's bits."""
    import threading
    server = es.exactsum_server_create(0, 64, 1 << 30, 1 << 16, 1 << 12)
    try:
        es.exactsum_server_set_lanes(server, 1 << 19, 8)
        out = {}
        lock = threading.Lock()

        def worker(seed):
            rng = np.random.default_rng(seed)
            for _ in range(60):
                dt = [es.F64, es.F32, es.BF16][int(rng.integers(0, 3))]
                bits, dx = pools[dt]
                n = int(rng.integers(0, 1 << int(rng.integers(4, 21))))
                o = int(rng.integers(0, len(bits) - n + 1))
                rid = es.exactsum_server_submit(server, dx[o:].data_ptr() if n else 0, n, dt, es.F64, es.RNE, 0)
                with lock:
                    out[rid] = (dt, o, n)

        threads = [threading.Thread(target=worker, args=(s,)) for s in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        recs = collect(server, len(out))
        assert len(recs) == len(out) == 240
        for rid, (dt, o, n) in out.items():
            assert recs[rid].status == es.OK
            assert recs[rid].result_bits == oracle.exact_sum(pools[dt][0][o:o + n], dt, es.F64, es.RNE, 2), rid
    finally:
        es.exactsum_server_destroy(server)


def test_destroy_while_resident_kernel_waits(pools):
    """Destroying a server right after its requests complete (the resident
    kernel still polling the queue) stops the kernel and returns; the device
    then runs other work normally."""
    bits, dx = pools[es.F64]
    for _ in range(3):
        server = es.exactsum_server_create(0, 8, 1 << 30, 1 << 15, 1 << 12)
        rid = es.exactsum_server_submit(server, dx.data_ptr(), 5000, es.F64, es.F64, es.RNE, 0)
        assert collect(server, 1)[rid].result_bits == oracle.exact_sum(bits[:5000], threads=2)
        es.exactsum_server_destroy(server)
    r = es.exact_sum(dx[:100_000])
    torch.cuda.synchronize()
    assert G.result_bits(r, es.F64)[0] == oracle.exact_sum(bits[:100_000], threads=2)
