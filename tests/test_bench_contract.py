"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one JSON
line with the keys and units of the benchmark contract, on the workload and metric
of the library arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def reference_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_line_keys(reference_line):
    l = reference_line
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in l, k
    assert l["impl"] == "reference" and l["unit"] == "GFLOP/s" and l["higher_is_better"] is True
    assert l["steps"] == 1 and l["warmup"] == 0 and l["n_gpus"] == 1 and l["value"] > 0
    assert l["data"] == "synthetic" and l["dtype"] == "f64"
    assert l["config"]["lattice"] == [16, 16, 16, 32] and l["config"]["Ls"] == 16


def test_reference_line_baseline_and_e2e(reference_line):
    cb, e2e = reference_line["cpu_baseline"], reference_line["e2e"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == reference_line["value"] and cb["sample"]
    assert e2e["value"] == reference_line["value"] and e2e["unit"] == reference_line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_metric_matches_library_arm(reference_line):
    sys.path.insert(0, ROOT)
    import bench
    assert reference_line["metric"] == bench.METRIC
    assert reference_line["config"] == bench.workload_config("f32")
