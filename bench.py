"""Benchmark: exact FP64 sum throughput on one GB300 (or N replicas).

Default workload: one FP64 array of n = 2^28 elements (2 GiB): (2^28 - 1024)/2
random-sign values with exponents uniform over [-1000, 1000] and uniform
52-bit fractions, their exact negations and 1024 uniform [-1, 1) residues,
shuffled with seed 0 (an ill-conditioned, delta ~ 2000 input).  One step is
one exact sum of the whole array, rounded to nearest-even FP64, through the
C ABI (``exactsum_sum``) with the input already resident in HBM.

Printed (rank 0, one JSON line): throughput in Gelem/s, the roofline of the
sum kernel against measured HBM bandwidth, the end-to-end figure through
``exactsum_sum_host`` from pinned host memory, the CPU oracle's throughput on
the host cores, and the SM clocks sampled during the timed region.  At N = 1
the line also carries, each measured after the headline's timed region:
the condition-number-sensitive path (``adaptive``); the 65,536-segment
batched sum against one launch per segment, every segment checked against
the oracle (``segmented``); the served request stream, an oracle sample,
alone-vs-mix re-submission and the one-launch-per-request baseline
(``serving``); the FP32 and BF16 single-array sums at full size
(``narrow``); and the exponent-range sweep over the four dataset families
(``delta_sweep``).

``--impl reference`` times the CPU oracle instead (the only baseline this
method has: the paper publishes no GPU or absolute numbers).

Multi-GPU: launched under torchrun, every rank sums its own array (weak
scaling, independent problems, no collective on the data path); the elapsed
time is the max over ranks.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("exact-sum Gelem/s and % of HBM roofline (FP64, 1×GB300); batched vs per-segment "
          "speedup; p99 latency")
WORKLOAD = ("single FP64 array, n = 2^28 (2 GiB): (2^28-1024)/2 random-sign values with exponent "
            "uniform in [-1000, 1000] and uniform 52-bit fraction, their exact negations, 1024 "
            "uniform [-1,1) residues, shuffled (seed 0); exact sum rounded to nearest-even FP64")
LOG2N = 28
BYTES_PER_ELEM = 8


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms), "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def sustained_clocks(torch, dev, stream, step, seconds=0.6):
    """The timed region is milliseconds long, shorter than nvidia-smi's
    sampling period, so its clock samples mostly see the GPU idle.  This
    repeats the same step back to back for about `seconds` right after the
    timed region, sampling clocks and throttle reasons every 50 ms, and
    reports them with the mean device time per step under that sustained
    load (untimed for the headline value)."""
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    per = max(a.elapsed_time(b), 0.01)
    reps = max(10, int(seconds * 1e3 / per))
    with ClockSampler(dev.index, period_ms=50) as clk:
        a.record(stream)
        for _ in range(reps):
            step()
        b.record(stream)
        torch.cuda.synchronize(dev)
    out = clk.summary()
    out["steps"] = reps
    out["ms_per_step"] = round(a.elapsed_time(b) / reps, 4)
    return out


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sum_kernel_tma_f64_traffic.json")
KERNEL_SOURCES = ["sum_kernels.cu", "sum_common.cuh", "stream.cuh", "digits.cuh", "tma.cuh", "finalize.cuh",
                  "internal.h"]
# the FP32 kernel (narrow block): the same sources as the FP64 one
TRAFFIC_FILE_F32 = os.path.join(ROOT, "profiles", "sum_kernel_f32_traffic.json")
# the BF16 FP32-digit kernel (narrow block)
TRAFFIC_FILE_BF16 = os.path.join(ROOT, "profiles", "sum_kernel_bf16t_traffic.json")
KERNEL_SOURCES_BF16 = ["sum_bf16.cu", "sum_common.cuh", "fdigits.cuh", "stream.cuh", "digits.cuh", "tma.cuh",
                       "finalize.cuh", "internal.h"]


def kernel_source_digest(sources=None) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, "paper_1605_05436_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(n, record=None, sources=None):
    """DRAM bytes per launch of a kernel from its committed ncu capture, or
    None when the kernel sources changed since it was taken or the size
    differs."""
    record = TRAFFIC_FILE if record is None else record
    if not os.path.exists(record):
        return None
    with open(record) as fh:
        d = json.load(fh)
    if d.get("kernel_sources_sha256") != kernel_source_digest(sources) or d.get("n") != n:
        return None
    return d.get("dram_bytes_per_launch")


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (empty if unknown)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return ""
    for ln in out.splitlines():
        if ln.strip().startswith("Model name:"):
            return ln.split(":", 1)[1].strip()
    return ""


def cpu_baseline(bits, passes: int, gpu_bits=None):
    """The CPU oracle, as it stands, on every host core (test infrastructure;
    timed here only as the reported baseline), plus a one-thread time on the
    first 2^24 elements.  When the GPU result is given, the oracle's result
    on the same full input is compared with it bit for bit."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.exact_sum(bits[: 1 << 16], threads=threads)  # load + warm
    t0 = time.perf_counter()
    for _ in range(passes):
        want = oracle.exact_sum(bits, threads=threads)
    dt = time.perf_counter() - t0
    one = bits[: 1 << 24]
    t1 = time.perf_counter()
    oracle.exact_sum(one, threads=1)
    dt1 = time.perf_counter() - t1
    out = {"value": round(passes * len(bits) / dt / 1e9, 4), "unit": "Gelem/s", "cores": threads,
           "kind": "oracle",
           "sample": f"the full 2^{LOG2N}-element workload, {passes} passes, {threads} threads "
                     f"({dt:.2f} s wall)",
           "cpu_model": cpu_model(),
           "single_thread": {"value": round(len(one) / dt1 / 1e9, 4), "unit": "Gelem/s",
                             "sample": "first 2^24 elements, 1 thread"}}
    if gpu_bits is not None:
        out["gpu_result_equals_oracle"] = (gpu_bits & ((1 << 64) - 1)) == want
    return out


# The paper's own measurements (Section 6.3), for context only: relative
# numbers from a CPU MapReduce (Spark) implementation; the paper prints no
# absolute times and no GPU figures, so there is no number to divide by.
PAPER_CONTEXT = {
    "source": "Goodrich & Eldawy, arXiv:1605.05436, Section 6.3 (experiments)",
    "hardware": "one AWS r3.8xlarge: 32 cores (Intel Xeon E5-2670 v2), 244 GB RAM; Spark 1.6.0 with 32 "
                "local workers on OpenJDK 1.7; baseline iFastSum in C++ (gcc 4.8.4)",
    "workload": "FP64, 1e6 to 1e9 numbers, exponent range delta = 2000 (10 to 2000 in a sweep), disk I/O not counted",
    "reported": "MapReduce with sparse or small superaccumulators up to 80x faster than sequential "
                "iFastSum; iFastSum faster below about 1e7 numbers; small accumulator slightly faster "
                "than sparse; linear scaling with cores up to 16, saturating from 16 to 32 (hyper-threads)",
    "absolute_times": None,
    "role": "context, not a target",
}


def naive_sum_context(torch, x, n, exact_bits, stream):
    """Context only: the plain FP64 tree reduction (torch.sum) on the same
    device array, its time and its error against the exact sum, in units in
    the last place of the exact result (as log2, since it can exceed the
    FP64 range)."""
    import struct
    from fractions import Fraction
    xf = x.view(torch.float64)
    for _ in range(3):
        r = xf.sum()
    torch.cuda.synchronize()
    times = []
    for _ in range(10):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = xf.sum()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    ms = times[len(times) // 2]
    naive = float(r.item())
    exact = struct.unpack("<d", struct.pack("<Q", exact_bits & ((1 << 64) - 1)))[0]
    out = {"impl": "torch.sum over the same FP64 array (library tree reduction, not exact)",
           "ms": round(ms, 4), "Gelem/s": round(n / ms / 1e6, 3), "result": repr(naive),
           "exact_result": repr(exact)}
    if math.isfinite(naive) and math.isfinite(exact):
        err = abs(Fraction(naive) - Fraction(exact))
        ulp = Fraction(math.ulp(exact))
        q = err / ulp
        out["log2_error_ulps"] = round(math.log2(q.numerator) - math.log2(q.denominator), 2) if err else None
    return out


def bench_segmented(es, W, torch, dev, steps, num_segments=65536, per_segment=True, check=True):
    """65,536 FP64 segments with log-uniform lengths in [1, 2^20] (Anderson-style
    mean-subtracted Gaussians scaled by 2^k, k uniform in [-200, 200]): the
    batched call (one graph-captured launch sequence, autotuned) against one
    exactsum_sum launch per segment, same results bit for bit; afterwards the
    CPU oracle checks the result of every segment of the timed launch."""
    lengths = W.segment_lengths(num_segments, seed=0)
    off = W.csr_offsets(lengths)
    total = int(off[-1])
    x = W.segmented_f64_device(lengths, seed=0, device=dev)
    d_off = torch.from_numpy(off).to(dev)
    h_off = torch.from_numpy(off)
    h = es.handle_for(dev.index)
    stream = torch.cuda.current_stream(dev)
    out_b = torch.empty(len(lengths), dtype=torch.float64, device=dev)
    out_e = torch.empty(len(lengths), dtype=torch.float64, device=dev)
    warps, kind, tile, tune_ms = es.exactsum_segmented_autotune(h, x.data_ptr(), d_off.data_ptr(), len(lengths),
                                                                es.F64, out_b.data_ptr(), stream.cuda_stream)

    def timed(fn, k):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / k

    batched_ms = timed(lambda: es.segmented_sum(x, d_off, out=out_b), max(3, steps))
    torch.cuda.synchronize(dev)
    batched_bits = out_b.view(torch.int64).cpu().numpy().view(np.uint64)
    if per_segment:
        each_ms = timed(lambda: es.sum_each(x, h_off, out=out_e), 2)
        same = bool(torch.equal(out_b.view(torch.int64), out_e.view(torch.int64)))
    else:
        each_ms, same = float("nan"), None
    t_chk = time.perf_counter()
    mism = oracle_check_segments(torch, x, off, batched_bits) if check else None
    t_chk = time.perf_counter() - t_chk
    r = {"workload": f"{num_segments:,} FP64 segments, lengths log-uniform [1, 2^20] (seed 0), N(0,1)*2^k, "
                     "k in [-200,200], minus the segment mean (device-generated)",
         "segments": len(lengths), "elements": total, "bytes": total * 8,
         "batched_ms": round(batched_ms, 3), "per_segment_ms": round(each_ms, 3) if per_segment else None,
         "speedup_vs_per_segment": round(each_ms / batched_ms, 2) if per_segment else None,
         "batched_gelem_s": round(total / batched_ms / 1e6, 2),
         "batched_hbm_gbs": round(total * 8 / batched_ms / 1e6, 1),
         "tuned": {"warps": warps, "reducer": ["register", "tma", "window"][kind], "tile": tile, "ms": round(tune_ms, 3)},
         "bit_identical_to_per_segment": same}
    if check:
        r["oracle_checked"] = len(lengths)
        r["oracle_mismatches"] = len(mism)
        r["oracle_first_mismatches"] = mism[:8]
        r["oracle_check"] = (f"every segment of the timed (autotuned) launch against the CPU oracle: input copied "
                             f"to the host in chunks of <= 2^27 elements, {os.cpu_count()} threads, {t_chk:.1f} s")
    del x
    torch.cuda.empty_cache()
    return r


def oracle_check_segments(torch, x, off, got_bits, chunk_elems=1 << 27):
    """Compare every segment's result bits with the CPU oracle (test
    infrastructure, run after the timed region).  The device input is
    copied to the host in chunks of whole segments; within a chunk the
    segments are spread over the host cores, one oracle thread each.
    Returns the indices of the segments that differ."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    threads = os.cpu_count() or 1
    S = len(off) - 1
    bad = []
    with ThreadPoolExecutor(threads) as pool:
        s = 0
        while s < S:
            e = s + 1
            while e < S and off[e + 1] - off[s] <= chunk_elems:
                e += 1
            lo, hi = int(off[s]), int(off[e])
            host = x[lo:hi].cpu().numpy().view(np.uint64)
            # groups of consecutive segments with about equal element counts
            rel = off[s:e + 1] - lo
            cuts = np.searchsorted(rel, np.linspace(0, hi - lo, threads + 1)[1:-1])
            bounds = sorted(set([0, *cuts.tolist(), e - s]))
            futs = [(a, pool.submit(oracle.exact_sum_segmented, host, rel[a:b + 1], 0, 0, 0, 1))
                    for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
            for a, f in futs:
                want = f.result().astype(np.uint64)
                got = got_bits[s + a:s + a + len(want)]
                bad.extend((np.nonzero(want != got)[0] + s + a).tolist())
            s = e
    return bad


def bench_serving(es, W, torch, dev, num_requests=100_000, chunk=1 << 21, max_steps=2, max_slots=128,
                  check=True, per_request=True, lanes=None):
    """Poisson stream of requests at 20k req/s (mean gap 50 us), sizes
    floor(2^(10 + 16U)), FP64 with p = 0.8 else FP32, windows into 2^26-element
    uniform [-1,1) device pools; served by the continuous-batching engine.

    Afterwards: the CPU oracle checks 1,000 random requests plus the 50
    largest; 100 sampled requests are submitted again, each alone, and must
    give the same bits; and the same stream, with the same arrival times, is
    replayed as one exactsum_sum launch per request (the baseline the engine
    is measured against), whose results must equal the served ones for
    every request."""
    if num_requests <= 0:
        return None
    req = W.serving_requests(num_requests, seed=0)
    pools = W.serving_pools(26, seed=0)
    d = {es.F64: torch.from_numpy(pools[es.F64].view(np.int64)).to(dev),
         es.F32: torch.from_numpy(pools[es.F32].view(np.int32)).to(dev)}
    base = {k: v.data_ptr() for k, v in d.items()}
    isz = {es.F64: 8, es.F32: 4}
    mask = {es.F64: (1 << 64) - 1, es.F32: (1 << 32) - 1}
    budget = 4 << 30
    ns, dts, offs, arr = (req["n"].tolist(), req["dtype"].tolist(), req["offset"].tolist(),
                          req["arrival_us"].tolist())
    N = len(ns)
    ids = [0] * N
    alone_mismatch = None
    alone_idx = np.random.default_rng(1).choice(N, min(100, N), replace=False).tolist()
    server = es.exactsum_server_create(dev.index, max_slots, budget, chunk, 1 << 15, max_steps)
    try:
        if lanes is not None:
            es.exactsum_server_set_lanes(server, *lanes)
        # warm the engine with a few requests
        for k in range(min(8, N)):
            es.exactsum_server_submit(server, base[dts[k]] + offs[k] * isz[dts[k]], ns[k], dts[k], dts[k], es.RNE, 0)
        es.exactsum_server_drain(server, 60_000)
        es.exactsum_server_poll(server)
        gc.disable()  # no collector pause inside the timed submission loop
        t0 = time.perf_counter()
        for k in range(N):
            target = arr[k] * 1e-6
            while time.perf_counter() - t0 < target:
                pass
            ids[k] = es.exactsum_server_submit(server, base[dts[k]] + offs[k] * isz[dts[k]], ns[k], dts[k],
                                               dts[k], es.RNE, 0)
        submit_span = time.perf_counter() - t0
        gc.enable()
        es.exactsum_server_drain(server, 600_000)
        recs = []
        while True:
            got = es.exactsum_server_poll(server, 65536)
            if not got:
                break
            recs.extend(got)
        stats = es.exactsum_server_stats(server)
        by_id = {r.id: r for r in recs}
        served = [by_id[i].result_bits & mask[dts[k]] if i in by_id else None for k, i in enumerate(ids)]
        if check:
            # the same request submitted alone gives the same bits
            alone_mismatch = 0
            for k in alone_idx:
                rid = es.exactsum_server_submit(server, base[dts[k]] + offs[k] * isz[dts[k]], ns[k], dts[k],
                                                dts[k], es.RNE, 0)
                es.exactsum_server_drain(server, 60_000)
                r = [c for c in es.exactsum_server_poll(server) if c.id == rid]
                if not r or (r[0].result_bits & mask[dts[k]]) != served[k]:
                    alone_mismatch += 1
    finally:
        es.exactsum_server_destroy(server)
    lat = np.array([r.done_ns - r.submit_ns for r in recs], dtype=np.float64) / 1e3
    ok = sum(1 for r in recs if r.status == es.OK)
    first = min(r.submit_ns for r in recs)
    last = max(r.done_ns for r in recs)
    elems = float(sum(ns))
    out = {"workload": "100,000 requests, Poisson 20k req/s, n = floor(2^(10+16U)), 80% FP64 / 20% FP32, "
                       "windows of 2^26-element uniform [-1,1) device pools (seed 0)",
           "requests": len(recs), "ok": ok, "offered_req_s": round(N / submit_span, 1),
           "p50_us": round(float(np.percentile(lat, 50)), 1), "p99_us": round(float(np.percentile(lat, 99)), 1),
           "mean_us": round(float(lat.mean()), 1), "max_us": round(float(lat.max()), 1),
           "gelem_s": round(elems / ((last - first) * 1e-9) / 1e9, 2),
           "engine": {"max_slots": max_slots, "budget_bytes": budget, "chunk_elems": chunk, "tile_elems": 1 << 15,
                      "max_steps_per_request": max_steps,
                      "lanes": {"express_max_bytes": lanes[0], "express_sms": lanes[1],
                                "resident": lanes[2] if len(lanes) > 2 else 1} if lanes else
                               "library defaults (express lane: requests up to 4 MiB of input, a resident "
                               "kernel on 8 SMs; bulk lane: one single-array launch per request on the "
                               "other SMs)",
                      "express_kernel_launches": stats["steps"], "peak_resident": stats["peak_active"]}}
    if check:
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        rng = np.random.default_rng(2)
        sample = set(rng.choice(N, min(1000, N), replace=False).tolist())
        sample |= set(np.argsort(np.asarray(ns), kind="stable")[-50:].tolist())
        sample = sorted(sample)
        threads = os.cpu_count() or 1
        t_chk = time.perf_counter()

        def want(k):
            return oracle.exact_sum(pools[dts[k]][offs[k]:offs[k] + ns[k]], dts[k], dts[k], es.RNE, 1)

        with ThreadPoolExecutor(threads) as pool:
            wants = list(pool.map(want, sample))
        bad = [k for k, w in zip(sample, wants) if served[k] != w]
        out["oracle_checked"] = len(sample)
        out["oracle_mismatches"] = len(bad)
        out["oracle_check"] = (f"{len(sample)} requests (1,000 uniformly sampled plus the 50 largest, "
                               f"{sum(ns[k] for k in sample) / 1e9:.2f}e9 elements) against the CPU oracle, "
                               f"{threads} threads, {time.perf_counter() - t_chk:.1f} s")
        out["alone_resubmitted"] = len(alone_idx)
        out["alone_mismatches"] = alone_mismatch
    if per_request:
        base_line = per_request_baseline(es, torch, dev, ns, dts, offs, arr, base, isz)
        res_bits = base_line.pop("_bits")
        diff = sum(1 for k in range(N) if served[k] != (int(res_bits[k]) & mask[dts[k]]))
        base_line["results_identical_to_served"] = diff == 0
        base_line["results_differing"] = diff
        out["per_request_baseline"] = base_line
        out["speedup_vs_per_request"] = {
            "p50": round(base_line["p50_us"] / out["p50_us"], 3),
            "p99": round(base_line["p99_us"] / out["p99_us"], 3),
            "gelem_s": round(out["gelem_s"] / base_line["gelem_s"], 3)}
    return out


def per_request_baseline(es, torch, dev, ns, dts, offs, arr, base, isz, ring=8192):
    """The serving workload without the engine: the same requests at the same
    arrival times, each summed by its own exactsum_sum launch on one stream
    (one handle), its completion observed through a CUDA event polled from
    the submitting loop.  Latency is launch -> event complete on the host."""
    import collections
    lib = es.library()
    h = es.handle_for(dev.index)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    N = len(ns)
    res = torch.zeros(N, dtype=torch.int64, device=dev)
    rp = res.data_ptr()
    fn = lib.exactsum_sum
    # warm: the first requests, and one request of every input format the
    # stream holds, so that no kernel is loaded inside the timed loop
    warm = list(range(min(8, N)))
    for d in sorted(set(int(v) for v in dts)):
        warm.append(next(k for k in range(N) if int(dts[k]) == d))
    for k in warm:
        fn(h, base[dts[k]] + offs[k] * isz[dts[k]], ns[k], dts[k], dts[k], es.RNE, rp + 8 * k, sp)
    torch.cuda.synchronize(dev)
    events = [torch.cuda.Event() for _ in range(ring)]
    sub = [0] * N
    done = [0] * N
    arr_ns = [int(a * 1e3) for a in arr]
    pending = collections.deque()
    pc = time.perf_counter_ns
    launches = 0
    gc.disable()  # no collector pause inside the timed loop (it would delay completions)
    t0 = pc()
    k = 0
    while k < N or pending:
        while pending and pending[0][1].query():
            j, _ = pending.popleft()
            done[j] = pc()
        if k < N and pc() - t0 >= arr_ns[k] and len(pending) < ring:
            sub[k] = pc()
            st = fn(h, base[dts[k]] + offs[k] * isz[dts[k]], ns[k], dts[k], dts[k], es.RNE, rp + 8 * k, sp)
            if st != es.OK:
                raise RuntimeError(f"exactsum_sum failed with status {st}")
            ev = events[k % ring]
            ev.record(stream)
            pending.append((k, ev))
            launches += 1
            k += 1
    gc.enable()
    torch.cuda.synchronize(dev)
    lat = (np.asarray(done, dtype=np.float64) - np.asarray(sub, dtype=np.float64)) / 1e3
    span = (max(done) - min(sub)) * 1e-9
    return {"impl": "one exactsum_sum launch per request, one stream and handle, same arrival times; "
                    "completion seen by polling a CUDA event per request",
            "launches": launches,
            "p50_us": round(float(np.percentile(lat, 50)), 1), "p99_us": round(float(np.percentile(lat, 99)), 1),
            "mean_us": round(float(lat.mean()), 1), "max_us": round(float(lat.max()), 1),
            "gelem_s": round(float(sum(ns)) / span / 1e9, 2),
            "_bits": res.cpu().numpy().view(np.uint64)}


def serving_isolated_latency(es, W, torch, dev, log2s=(10, 14, 16, 18, 20, 22, 24, 26), reps=200, lanes=None):
    """Latency of lone FP64 requests (one at a time, 100 us apart, median of
    `reps`): one exactsum_sum launch with a CUDA event polled from the host,
    against the serving engine (with the given lanes, else its defaults)."""
    pool = torch.from_numpy(W.uniform_f64(1 << max(log2s), 0).view(np.int64)).to(dev)
    base = pool.data_ptr()
    lib = es.library()
    h = es.handle_for(dev.index)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    res = torch.zeros(1, dtype=torch.int64, device=dev)
    ev = torch.cuda.Event()

    def pause():
        t1 = time.perf_counter_ns()
        while time.perf_counter_ns() - t1 < 100_000:
            pass

    rows = []
    for lg in log2s:
        n = 1 << lg
        lat = []
        for _ in range(reps):
            t0 = time.perf_counter_ns()
            lib.exactsum_sum(h, base, n, es.F64, es.F64, es.RNE, res.data_ptr(), sp)
            ev.record(stream)
            while not ev.query():
                pass
            lat.append(time.perf_counter_ns() - t0)
            pause()
        direct = float(np.median(lat)) / 1e3
        s = es.exactsum_server_create(dev.index, 128, 4 << 30, 1 << 21, 1 << 15, 2)
        try:
            if lanes is not None:
                es.exactsum_server_set_lanes(s, *lanes)
            lat = []
            for _ in range(reps):
                es.exactsum_server_submit(s, base, n, es.F64, es.F64, es.RNE, 0)
                while True:
                    got = es.exactsum_server_poll(s, 16)
                    if got:
                        break
                lat.append(got[0].done_ns - got[0].submit_ns)
                pause()
        finally:
            es.exactsum_server_destroy(s)
        rows.append({"log2n": lg, "one_launch_us": round(direct, 1), "engine_us": round(float(np.median(lat)) / 1e3, 1)})
    return rows


def run_serving(args):
    """The serving measurement alone, with chosen lanes (profiling runs)."""
    import torch

    import paper_1605_05436_gb300 as es
    from paper_1605_05436_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    es.build()
    lanes = tuple(int(v) for v in args.lanes.split(",")) if args.lanes else None
    line = {"metric": "served exact sums: latency and throughput (profiling case)",
            "lanes": args.lanes or "library defaults"}
    if args.isolated_latency:
        line["isolated"] = serving_isolated_latency(es, W, torch, dev, lanes=lanes)
    else:
        line["serving"] = bench_serving(es, W, torch, dev, args.requests, check=not args.no_check,
                                        per_request=not args.no_per_request, lanes=lanes)
    print(json.dumps(line), flush=True)
    return 0


def bench_adaptive(es, torch, dev, x, n, reps=3):
    """The condition-number-sensitive path (r-truncated passes, r <- r^2)
    beside the exact single pass, on the benchmark input and on a
    well-conditioned one of the same size: passes needed and wall time of
    the synchronous call (median of ``reps`` after one warm-up)."""
    h = es.handle_for(dev.index)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize(dev)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts) * 1e3, r

    res = {}
    uni = (torch.rand(n, dtype=torch.float64, device=dev) * 2 - 1).view(torch.int64)
    for name, arr in (("cancelling delta~2000 (the benchmark input)", x),
                      ("uniform [-1,1) (device-generated)", uni)):
        ms_a, (passes, last_r) = timed(lambda: es.exactsum_sum_adaptive(
            h, arr.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(), s))
        bits_a = int(out.view(torch.int64).item())
        ms_e, _ = timed(lambda: es.exactsum_sum(h, arr.data_ptr(), n, es.F64, es.F64, es.RNE,
                                                out.data_ptr(), s))
        bits_e = int(out.view(torch.int64).item())
        res[name] = {"passes": passes, "last_r": last_r, "adaptive_ms": round(ms_a, 3),
                     "exact_ms": round(ms_e, 3), "same_result": bits_a == bits_e}
    del uni
    return {"n": n, "api": "exactsum_sum_adaptive (synchronous; r = 2, 4, 16, then the exact pass)",
            "workloads": res}


def run_delta_sweep(args):
    """Throughput of the FP64 exact sum over the paper's four dataset families
    and exponent ranges delta (the design of the paper's Fig. 2 experiment,
    on this GPU): the dense accumulator's cost should not depend on delta."""
    import torch
    import paper_1605_05436_gb300 as es
    from paper_1605_05436_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    es.build()
    n = 1 << args.log2n
    h = es.handle_for(0)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev)
    rows = []
    for family in (1, 2, 3, 4):
        for delta in (10, 100, 500, 1000, 2000, 2046):
            bits = W.family_f64(family, n, delta, seed=family)
            x = torch.from_numpy(bits.view(np.int64)).to(dev)
            for _ in range(3):
                es.exactsum_sum(h, x.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(), s.cuda_stream)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(args.steps):
                es.exactsum_sum(h, x.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(), s.cuda_stream)
            b.record(s)
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / args.steps
            rows.append({"family": family, "delta": delta, "ms": round(ms, 4),
                         "gelem_s": round(n / ms / 1e6, 1), "gb_s": round(8 * n / ms / 1e6, 1)})
            del x
    peak, kind = measured_peaks()
    line = {"metric": "exact-sum Gelem/s vs exponent range delta, four dataset families (FP64, 1xGB300)",
            "unit": "Gelem/s", "n": n, "steps": args.steps, "higher_is_better": True, "data": "synthetic",
            "families": {"1": "all positive", "2": "mixed signs", "3": "mixed signs minus the mean",
                         "4": "exact sum zero (+/- pairs)"},
            "peak_gb_s": peak, "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    from paper_1605_05436_gb300 import workloads as W
    import oracle
    n = 1 << args.log2n
    bits = W.cancelling_f64(n, seed=0)
    threads = os.cpu_count() or 1
    # each step: one pass of the oracle over a bounded sample of the workload
    sample = bits[: 1 << min(26, args.log2n)]
    for _ in range(args.warmup):
        oracle.exact_sum(sample, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.exact_sum(sample, threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * len(sample) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Gelem/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.log2n == LOG2N
                   else f"profiling case: n = 2^{args.log2n}, same recipe",
                   "n": n, "sample_per_step": len(sample)},
        "cpu_baseline": {"value": round(value, 4), "unit": "Gelem/s", "cores": threads,
                         "kind": "oracle",
                         "sample": f"first {len(sample)} elements of the workload per step, "
                                   f"{threads} threads"},
        "e2e": {"value": round(value, 4), "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# The integer-ALU pipe of one sub-partition issues one warp instruction every
# two cycles (16 lanes per cycle): 152 SMs x 4 sub-partitions x 16 lanes x the
# SM clock is the ALU roof of the kernels that integer decoding binds.
ALU_LANES_PER_SM_CYCLE = 64


def bench_narrow(es, W, torch, dev, dt, steps, warmup, log2n=None, check=True):
    """FP32 or BF16 single-array exact sum on the wide-exponent recipes
    (FP32: n = 2^29, 99% normals with biased exponent uniform in [1, 254] and
    1% subnormals; BF16: n = 2^30, exponent uniform in [-126, 127]), rounded
    to the input format: device time per launch (CUDA events on the launching
    stream, inputs of 2 GiB > L2), HBM roofline, clocks, and the result
    checked against the CPU oracle on the full input."""
    name = "f32" if dt == es.F32 else "bf16"
    log2n = log2n if log2n is not None else (29 if dt == es.F32 else 30)
    n = 1 << log2n
    eb = 4 if dt == es.F32 else 2
    t_gen = time.perf_counter()
    bits = W.wide_f32(n, seed=0) if dt == es.F32 else W.wide_bf16(n, seed=0)
    t_gen = time.perf_counter() - t_gen
    x = torch.from_numpy(bits.view(np.int32 if dt == es.F32 else np.int16)).to(dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = es.handle_for(dev.index)
    for _ in range(max(warmup, 3)):
        es.exactsum_sum(h, x.data_ptr(), n, dt, dt, es.RNE, out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(dev)
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clocks:
        t_begin.record(stream)
        for i in range(steps):
            es.exactsum_sum(h, x.data_ptr(), n, dt, dt, es.RNE, out.data_ptr(), stream.cuda_stream)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    ms = t_begin.elapsed_time(t_end) / steps  # back-to-back launches, two events around them
    peak, peak_kind = measured_peaks()
    achieved = n * eb / (ms * 1e-3) / 1e9
    result_bits = int(out.view(torch.int64).item()) & ((1 << (8 * eb)) - 1)
    clk = clocks.summary()
    sustained = sustained_clocks(torch, dev, stream, lambda: es.exactsum_sum(
        h, x.data_ptr(), n, dt, dt, es.RNE, out.data_ptr(), stream.cuda_stream))
    sm_mhz = clk.get("sm_mhz") or 2070.0
    alu_roof = es_sm_count(torch, dev) * ALU_LANES_PER_SM_CYCLE * sm_mhz * 1e6
    r = {"workload": f"{name.upper()} n = 2^{log2n}, wide-exponent recipe (seed 0), rounded to the input format",
         "n": n, "launches": steps, "ms": round(ms, 4), "gelem_s": round(n / ms / 1e6, 1),
         "roofline": {"bound": NARROW_BOUND[name], "hbm_achieved": round(achieved, 1), "hbm_peak": peak,
                      "unit": "GB/s", "hbm_frac": round(achieved / peak, 4),
                      "peak_kind": f"{peak_kind} (STREAM-style copy)",
                      "algorithmic_bytes_per_launch": n * eb,
                      "traffic": (measured_traffic(n, TRAFFIC_FILE_BF16, KERNEL_SOURCES_BF16)
                                  if dt == es.BF16 else measured_traffic(n, TRAFFIC_FILE_F32, KERNEL_SOURCES)),
                      "alu_roof_tera_lane_ops_per_s": round(alu_roof / 1e12, 2),
                      "alu_roof": "SMs x 4 sub-partitions x 16 ALU lanes per cycle x median SM clock; "
                                  "instructions per element from ncu are in profiles/"},
         "clocks": clk, "clocks_sustained": sustained, "result_bits": f"{result_bits:#x}"}
    if check:
        import oracle
        # the wide recipes' sums overflow the input format (the rounded result
        # is an infinity), so the exact sum is also rounded to FP64, untimed,
        # where every element counts, and compared too
        es.exactsum_sum(h, x.data_ptr(), n, dt, es.F64, es.RNE, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        f64_bits = int(out.view(torch.int64).item()) & ((1 << 64) - 1)
        t_chk = time.perf_counter()
        want = oracle.exact_sum(bits, dt, dt, es.RNE, threads=os.cpu_count() or 1)
        want64 = oracle.exact_sum(bits, dt, es.F64, es.RNE, threads=os.cpu_count() or 1)
        r["gpu_result_equals_oracle"] = result_bits == want
        r["result_f64_bits"] = f"{f64_bits:#x}"
        r["gpu_f64_result_equals_oracle"] = f64_bits == want64
        r["oracle_check"] = (f"full input, rounded to the input format and to FP64, {os.cpu_count()} threads, "
                             f"{time.perf_counter() - t_chk:.1f} s (input generated in {t_gen:.1f} s)")
    del x
    torch.cuda.empty_cache()
    return r


# What bounds each narrow-format kernel (from ncu): FP32 keeps the integer ALU
# pipe 82 % busy; the BF16 FP32-digit kernel leaves it at 63 % and streams at
# 81 % of HBM bandwidth, near issue-bound, so its roof is the HBM one.
NARROW_BOUND = {"f32": "alu", "bf16": "hbm"}


def es_sm_count(torch, dev) -> int:
    return torch.cuda.get_device_properties(dev).multi_processor_count


def bench_delta_block(es, W, torch, dev, log2n=26, deltas=(10, 2000, 2046), steps=20, check=True):
    """A compact form of the delta sweep (the design of the paper's Fig. 2,
    Section 6.3) on the benchmark kernel: the four dataset families at three
    exponent ranges, n = 2^26 FP64 (512 MiB, larger than L2), device time per
    launch and, for each input, the result against the CPU oracle."""
    n = 1 << log2n
    h = es.handle_for(dev.index)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev)
    peak, _ = measured_peaks()
    rows = []
    mism = 0
    for family in (1, 2, 3, 4):
        for delta in deltas:
            bits = W.family_f64(family, n, delta, seed=family)
            x = torch.from_numpy(bits.view(np.int64)).to(dev)
            for _ in range(3):
                es.exactsum_sum(h, x.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(), s.cuda_stream)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(steps):
                es.exactsum_sum(h, x.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(), s.cuda_stream)
            b.record(s)
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / steps
            row = {"family": family, "delta": delta, "ms": round(ms, 4), "gelem_s": round(n / ms / 1e6, 1),
                   "hbm_frac": round(8 * n / ms / 1e6 / peak, 4)}
            if check:
                import oracle
                got = int(out.view(torch.int64).item()) & ((1 << 64) - 1)
                row["equals_oracle"] = got == oracle.exact_sum(bits, threads=os.cpu_count() or 1)
                mism += 0 if row["equals_oracle"] else 1
            rows.append(row)
            del x
    return {"n": n, "launches_per_row": steps,
            "families": {"1": "all positive", "2": "mixed signs", "3": "mixed signs minus the mean",
                         "4": "exact sum zero (+/- pairs)"},
            "kernel": "the benchmark kernel (exactsum_sum, FP64 -> FP64, RNE)",
            "rows": rows, "oracle_mismatches": mism if check else None}


def run_narrow(args):
    """The FP32 / BF16 line alone (profiling runs)."""
    import torch

    import paper_1605_05436_gb300 as es
    from paper_1605_05436_gb300 import workloads as W

    dt = {"f32": es.F32, "bf16": es.BF16}[args.dtype]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    es.build()
    r = bench_narrow(es, W, torch, dev, dt, args.steps, args.warmup, args.log2n, check=not args.no_check)
    line = {"metric": f"exact-sum Gelem/s ({args.dtype.upper()}, profiling case)",
            "value": r["gelem_s"], "unit": "Gelem/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
            "dtype": "int64" if dt == es.F32 else "int32", "data": "synthetic",
            "config": {"workload": r["workload"], "launch": "exactsum_sum, one kernel per step"},
            "roofline": r["roofline"], "gpu_launches": args.steps, "clocks": r["clocks"],
            "clocks_sustained": r["clocks_sustained"], "result_bits": r["result_bits"]}
    if "gpu_result_equals_oracle" in r:
        line["gpu_result_equals_oracle"] = r["gpu_result_equals_oracle"]
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1605_05436_gb300 as es
    from paper_1605_05436_gb300 import workloads as W

    ws, rank, local = dist_info()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    es.build()
    n = 1 << args.log2n
    bits = W.cancelling_f64(n, seed=rank)
    x = torch.from_numpy(bits.view(np.int64)).to(dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = es.handle_for(local)
    sptr = stream.cuda_stream

    def step():
        es.exactsum_sum(h, x.data_ptr(), n, es.F64, es.F64, es.RNE, out.data_ptr(), sptr)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    # the K launches run back to back on the launching stream, bracketed by
    # two CUDA events only (an event between two launches would stop the next
    # one from starting while the one before merges and rounds)
    with ClockSampler(local) as clocks:
        t_begin = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_begin.record(stream)
        for i in range(args.steps):
            step()
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    elapsed_ms = t_begin.elapsed_time(t_end)
    local_elapsed_ms = elapsed_ms
    if ws > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    result_bits = int(out.view(torch.int64).item())

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        h_x = torch.from_numpy(bits.view(np.int64)).pin_memory()
        es.exact_sum_host(h_x)
        torch.cuda.synchronize(dev)
        e2e_steps = max(2, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_bits = es.exact_sum_host(h_x)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        assert e2e_bits == result_bits & ((1 << 64) - 1), "end-to-end result differs from device result"
        if ws > 1:  # whole-job time: the slowest rank
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": round(ws * n / e2e_s / 1e9, 3), "unit": "Gelem/s",
               "h2d_bytes_per_step": n * BYTES_PER_ELEM, "d2h_bytes_per_step": 8,
               "api": "exactsum_sum_host (pinned host buffer, 64 MiB chunks, copy/compute overlap)",
               "steps": e2e_steps}

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    ms_per_step = elapsed_ms / args.steps
    value = ws * n / (ms_per_step * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    avg_kernel_ms = local_elapsed_ms / args.steps  # one launch per step, back to back
    achieved = n * BYTES_PER_ELEM / (avg_kernel_ms * 1e-3) / 1e9
    traffic = measured_traffic(n)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gelem/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "in": "f64", "out": "f64", "mode": "rne",
                   "per_rank": "independent array per rank (seed = rank)",
                   "l2": "input 2 GiB > 129 MB L2 between steps; no flush needed",
                   "launch": "exactsum_sum, one kernel per step"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "frac_of_nominal_8000_gbs": round(achieved / 8000.0, 4),
                     "peak_kind": f"{peak_kind} (STREAM-style copy)",
                     "kernel": "es::sum_kernel_tma<F64, 8 consumer warps, 10 vectors per thread per stage, 2 stages>",
                     "algorithmic_bytes_per_launch": n * BYTES_PER_ELEM,
                     "avg_kernel_ms": round(avg_kernel_ms, 4),
                     "avg_kernel_ms_is": "CUDA events around the K back-to-back launches of the timed region, "
                                         "elapsed / K (a launch may start while the one before it merges and "
                                         "rounds: programmatic dependent launch)"},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks.summary(),
        "clocks_sustained": sustained_clocks(torch, dev, stream, step),
        "result_bits": f"{result_bits & ((1 << 64) - 1):#018x}",
    }
    if args.log2n != LOG2N:
        line["config"]["workload"] = f"profiling case: n = 2^{args.log2n}, same recipe"
    line["context"] = {"naive_fp64_sum": naive_sum_context(torch, x, n, result_bits, stream),
                       "paper": PAPER_CONTEXT}
    if not args.no_cpu_baseline and ws == 1:  # the oracle is timed at N = 1 only
        line["cpu_baseline"] = cpu_baseline(bits, passes=8, gpu_bits=result_bits)
    if ws == 1 and (args.adaptive or (args.log2n == LOG2N and not args.primary_only)):
        line["adaptive"] = bench_adaptive(es, torch, dev, x, n)
    if ws == 1 and args.log2n == LOG2N and not args.primary_only:
        del x
        torch.cuda.empty_cache()
        line["segmented"] = bench_segmented(es, W, torch, dev, args.steps, args.segments,
                                            not args.no_per_segment, check=not args.no_check)
        line["serving"] = bench_serving(es, W, torch, dev, args.requests, check=not args.no_check,
                                        per_request=not args.no_per_request)
        if not args.no_narrow:
            line["narrow"] = {"f32": bench_narrow(es, W, torch, dev, es.F32, args.steps, args.warmup,
                                                  check=not args.no_check),
                              "bf16": bench_narrow(es, W, torch, dev, es.BF16, args.steps, args.warmup,
                                                   check=not args.no_check)}
        if not args.no_delta:
            line["delta_sweep"] = bench_delta_block(es, W, torch, dev, check=not args.no_check)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--primary-only", action="store_true",
                    help="skip the segmented and serving measurements")
    ap.add_argument("--segments", type=int, default=65536,
                    help="segments of the batched measurement (65,536 is the benchmark workload)")
    ap.add_argument("--no-per-segment", action="store_true",
                    help="skip the one-launch-per-segment baseline (profiling runs)")
    ap.add_argument("--delta-sweep", action="store_true",
                    help="print the exponent-range sweep over the four dataset families instead")
    ap.add_argument("--requests", type=int, default=100_000,
                    help="requests of the serving measurement (0 skips it)")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the CPU-oracle checks after the timed regions (profiling runs)")
    ap.add_argument("--no-per-request", action="store_true",
                    help="skip the one-launch-per-request serving baseline")
    ap.add_argument("--no-narrow", action="store_true", help="skip the FP32/BF16 block of the default line")
    ap.add_argument("--no-delta", action="store_true", help="skip the delta-sweep block of the default line")
    ap.add_argument("--serving-only", action="store_true",
                    help="print only the serving measurement (profiling runs)")
    ap.add_argument("--lanes", default=None,
                    help="with --serving-only: EXPRESS_MAX_BYTES,EXPRESS_SMS,RESIDENT for exactsum_server_set_lanes")
    ap.add_argument("--isolated-latency", action="store_true",
                    help="with --serving-only: lone requests of 2^10..2^26 elements, engine against one launch")
    ap.add_argument("--adaptive", action="store_true",
                    help="also time the condition-number-sensitive path with --primary-only or --log2n")
    ap.add_argument("--dtype", choices=["f64", "f32", "bf16"], default="f64",
                    help="f32/bf16: profiling line for the narrow formats instead of the benchmark")
    ap.add_argument("--log2n", type=int, default=None,
                    help="smaller cases for profiling only; the benchmark line uses 2^28")
    args = ap.parse_args()
    if args.log2n is None and (args.dtype == "f64" or args.impl == "reference"):
        args.log2n = LOG2N
    if args.impl == "reference":
        return run_reference(args)
    if args.delta_sweep:
        return run_delta_sweep(args)
    if args.serving_only:
        return run_serving(args)
    if args.dtype != "f64":
        return run_narrow(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
