"""bench.py's reference arm (the CPU oracle timed on the host) prints the one
JSON line the benchmark contract asks for; runs without a GPU."""
import json
import os
import subprocess
import sys

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_json_line():
    import bench
    line = _run("--impl", "reference", "--steps", "2", "--warmup", "3", "--bytes", str(1 << 20))
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "GB/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] >= 3 and line["n_gpus"] == 1
    assert line["config"]["workload"].startswith("regex512_")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_workload_size_names():
    assert gen._size_name(1 << 30) == "1GiB"
    assert gen._size_name(10 * 10**9) == "10GB"
    assert gen._size_name(4 << 20) == "4MiB"
    assert gen._size_name(12345) == "12345B"
