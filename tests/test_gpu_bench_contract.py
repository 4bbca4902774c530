"""The benchmark's JSON line on a GPU: one line with the keys and value types the measurement
contract names (throughput, roofline of the dominant kernel, end-to-end figures with the bytes
copied each step, clock record, launch count), from a short run of the default workload."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3", "--no-extras",
           "--no-cpu-baseline", "--launch", "64,16,32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and "workload" in d["config"]
    roof = d["roofline"]
    assert roof["bound"] in ("hbm", "tensor", "alu") and roof["unit"] in ("GB/s", "TFLOP/s")
    assert roof["achieved"] > 0 and roof["peak"] > 0 and abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-3
    assert "traffic" in roof
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == d["unit"]
    n, m, k = d["config"]["n"], d["config"]["m"], d["config"]["k"]
    assert e2e["h2d_bytes_per_step"] == 12 * (n + m)  # points and queries, float32 xyz
    assert e2e["d2h_bytes_per_step"] >= 8 * (m + 1) + 8 * m * k  # offsets, k-NN rows and distances, CSR rows
    assert d["gpu_launches"] >= 10
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
