"""CPU checks of bench.py's contract: the reference arm (the CPU oracle)
prints one JSON line with the keys the benchmark line promises, ranks other
than 0 print nothing, and the host-side helpers behave."""
from __future__ import annotations

import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_reference_arm_line():
    lines = run_bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--log2n", "16"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Gelem/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["n"] == 1 << 16 and "profiling case" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent():
    lines = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--log2n", "12"],
                      {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


def test_traffic_record_is_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    rec = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.measured_traffic(1 << 28) is None  # no record
    rec.write_text(json.dumps({"kernel_sources_sha256": bench.kernel_source_digest(), "n": 1 << 28,
                               "dram_bytes_per_launch": 123}))
    assert bench.measured_traffic(1 << 28) == 123
    assert bench.measured_traffic(1 << 20) is None  # another size
    rec.write_text(json.dumps({"kernel_sources_sha256": "0" * 64, "n": 1 << 28,
                               "dram_bytes_per_launch": 123}))
    assert bench.measured_traffic(1 << 28) is None  # sources changed since the capture


def test_clock_summary_flags_throttling():
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1900, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    d = s.summary()
    assert d["samples"] == 3 and d["sm_mhz"] == 2070 and d["sm_max_mhz"] == 2070
    assert d["reasons"] == ["sw_power_cap"]
    s.lines = ["0, 1200, 2070, 700, 0x8, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary()["reasons"] == ["unavailable"]


def test_segment_check_finds_every_planted_mismatch():
    """The bench's full oracle check of the segmented results (run here on a
    CPU tensor): correct bits pass, and each altered result is reported,
    across chunk and thread-group boundaries."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch

    import bench
    import oracle
    from paper_1605_05436_gb300 import workloads as W
    lengths = W.segment_lengths(300, seed=3, log2_max=12)
    lengths[::11] = 0
    off = W.csr_offsets(lengths)
    bits = W.segmented_f64(lengths, seed=4)
    x = torch.from_numpy(bits.view(np.int64))
    good = oracle.exact_sum_segmented(bits, off, threads=2).astype(np.uint64)
    assert bench.oracle_check_segments(torch, x, off, good, chunk_elems=5000) == []
    bad = good.copy()
    planted = [0, 17, 150, 299]
    for s in planted:
        bad[s] ^= np.uint64(1)
    assert bench.oracle_check_segments(torch, x, off, bad, chunk_elems=5000) == planted
    assert bench.oracle_check_segments(torch, x, off, bad, chunk_elems=1 << 30) == planted
