"""Host-side checks of bench.py: the algorithmic byte model, the clock-reason
decoding, the traffic lookup's source-hash guard, max-over-ranks timing with
two gloo processes, and the reference arm (rank 0 prints one JSON line, other
ranks exit without work) on the small workload."""
import hashlib
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_bytes_model():
    n, m, k, nnz = 10_000_000, 1_000_000, 10, 9_930_677
    nodes = {"spatial": 66_540_000, "nearest": 78_860_000}
    assert bench.kernel_bytes("bounds", n, m, k, nnz, nodes) == 12 * n
    assert bench.kernel_bytes("nearest", n, m, k, nnz, nodes) == m * (16 + 8 * k + 8) + 64 * nodes["nearest"]
    # 30-bit keys: 4 passes; the first reads keys only (12 B/key), later passes move pairs (16 B/key)
    assert bench.kernel_bytes("onesweep_pass", n, m, k, nnz, nodes) == (n + m) * (12 + 16 * 3)
    assert bench.kernel_bytes("apetrei", n, m, k, nnz, nodes) == 52 * n + 32 * (n - 1)
    assert bench.kernel_bytes("spatial_buffered", n, m, k, nnz, nodes) == 20 * m + 4 * nnz + 64 * nodes["spatial"]
    assert bench.kernel_bytes("no_such_kernel", n, m, k, nnz, nodes) is None


def test_clock_summary_decodes_reasons():
    c = bench.ClockSampler(0)
    c.max_mhz = 2032.0
    c.samples = [(2032.0, 0), (2010.0, 0x4), (1980.0, 0x4 | 0x40), (2032.0, 0x1)]
    s = c.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == pytest.approx(2021.0)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]  # 0x1 (idle) is not a throttle reason
    assert bench.ClockSampler(0).summary()["sm_mhz"] is None


def test_measured_traffic_requires_matching_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"nearest": {"dram_bytes": 123, "file": "k.cu", "csrc_sha": sha, "workload": "cube_1e7"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("nearest", "cube_1e7") == 123
    assert bench.measured_traffic("nearest", "cube_1e6") is None  # another workload
    assert bench.measured_traffic("compact", "cube_1e7") is None  # never captured
    src.write_text("kernel source v2\n")  # the kernel changed since the capture
    assert bench.measured_traffic("nearest", "cube_1e7") is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        out[rank] = bench.max_over_ranks(1.5 + rank, ws, "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_max_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: 2.5, 1: 2.5}  # every rank sees the slowest rank's time
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0


def test_reference_arm_rank0_only_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "cube_1e4", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 1 exits without work or output
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
