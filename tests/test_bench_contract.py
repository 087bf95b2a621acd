"""bench.py's reference arm (the oracle on the host cores) prints one JSON line with the
keys of the benchmark contract; the byte models match their stated formulas."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_default_workload_is_the_headline_config():
    # with no flags, bench.py measures R-MAT scale 24 with k = 8192 sampled sources
    import bench
    saved = sys.argv
    try:
        sys.argv = ["bench.py"]
        args = bench.parse()
    finally:
        sys.argv = saved
    assert args.config == "rmat24" and args.gpus == 1 and args.warmup >= 3
    cfg = bench.CONFIGS[args.config]
    assert (cfg["kind"], cfg["size"], cfg["k"]) == ("rmat", 24, 8192)


def test_reference_arm_json_line():
    # the contract's keys do not depend on the workload: the small config keeps this quick
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--config", "rmat18", "--steps", "1", "--warmup", "0"], capture_output=True,
                         text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "GTEPS" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0


def test_byte_models():
    import bench
    n, A = 1000, 16000
    assert bench.algorithmic_bytes_per_launch(n, A, 64) == 8 * A + 24 * n + 34 * n * 64
    assert bench.per_source_bytes(n, A) == 8 * A + 64 * n
    assert bench.edge_bytes(n, A, 128) == 8 * A + 24 * n + 34 * n * 128 + 16 * A
    assert bench.rk_bytes(n, A, 128) == 4 * A + 12 * n + 17 * n * 128
    assert bench.closeness_bytes(n, A, 128, 5) == 4 * A + 12 * n + 17 * n * 128 + 8 * n * 2 * 5 + 32 * n
    assert bench.weighted_bytes(n, A) == 16 * A + 56 * n
    r = bench._roof(1e9, 2.0, 1000.0, "measured", "k")
    assert abs(r["achieved"] - 500.0) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12


def test_committed_traffic_follows_kernel_sources():
    # the committed DRAM traffic is reported only while the kernel sources hash as captured
    # (after a kernel change it reads null until the capture is repeated)
    import bench
    pj = json.load(open(os.path.join(ROOT, "profiles", "k_batch_rmat24_traffic.json")))
    current = pj["kernel_source_sha256"] == bench.kernel_source_hash(pj["kernel_sources"])
    want = pj["by_batch"]["128"]["dram_bytes_per_launch"] if current else None
    assert bench.committed_traffic("rmat24", 128, False) == want
    assert bench.committed_traffic("rmat24", 64) is None
    assert bench.committed_traffic("rmat24", 128, True) is None
