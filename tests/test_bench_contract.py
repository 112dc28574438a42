"""bench.py's reference arm (the CPU oracle on a bounded sample of the headline workload)
prints one JSON line with the keys the benchmark contract names; runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--ref-budget", "200000"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "chunglu1m_top100_cliques"


def test_serving_latency_quantiles():
    """The serving line's p50/p99 (overall and per request kind): nearest rank on the sorted
    latencies, None for a kind with no requests."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench._pct([], 0.5) is None
    v = list(range(100, 0, -1))  # 1..100, unsorted
    assert bench._pct(v, 0.5) == 51 and bench._pct(v, 0.99) == 100
    assert bench._pct([3.0, 1.0, 2.0], 0.0) == 1.0 and bench._pct([7.0], 0.99) == 7.0
