"""Benchmark of the LBVH search path on B300.

One step = the whole hot path over one batch of synthetic input: build the
tree over n points (scene box, Morton codes, radix sort, hierarchy and box
fit), Morton-sort the queries once, then the spatial query and the k-nearest
query, in that order.  The spatial query is the one-call one-pass form (rows
into a per-query buffer of the tuner's width, overflowing rows refilled, no
host round trip) when the tuner picks a buffer width, else the two-pass form
(count, scan, read the total, fill).  Default workload: n = 1e7 points uniform
in the unit cube, m = 1e6 queries from the same distribution, radius for a
mean of 10 neighbours, k = 10.

Prints one JSON line (rank 0).  `value` is the query throughput of the whole
step in Mqueries/s (radius + nearest queries per second of build+query time),
with inputs resident in HBM; `e2e` is the same metric with the points and
queries copied from pinned host memory and all results copied back inside the
timed region.  L2 is flushed between timed steps (a 256 MB write, then a 256 MB
read of a second buffer).

--impl reference times the CPU oracle (median-split CPU BVH, OpenMP) on the
host cores over the same workload: each step builds its tree over all points
and runs all m radius and m nearest queries (``--ref-queries`` times fewer);
the line reports what was measured, nothing is extrapolated.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

METRIC = "kNN k=10 & radius Mqueries/s + build Mpts/s at 1e7 pts; learned vs plain"
UNIT = "Mqueries/s"

WORKLOADS = {
    # name: (distribution, n, m, k)
    "cube_1e7": ("cube", 10_000_000, 1_000_000, 10),
    "hollow_sphere_1e7": ("hollow_sphere", 10_000_000, 1_000_000, 10),
    "cube_1e6": ("cube", 1_000_000, 1_000_000, 10),
    "cube_1e4": ("cube", 10_000, 10_000, 10),  # the small oracle-sized case (host tests)
}


# ---------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """Largest value of x over all ranks (the slowest rank's time); x itself when ws == 1."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (SM clock, maximum SM clock,
    current clock-event reasons)."""

    def __init__(self, index: int):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex failed")
        try:
            self._reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self._reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _clock(self, fn) -> float:
        v = self.c.c_uint()
        if fn(self.h, self.c.c_int(1), self.c.byref(v)) != 0:  # NVML_CLOCK_SM
            raise RuntimeError("nvml clock query failed")
        return float(v.value)

    def sm_mhz(self) -> float:
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def max_sm_mhz(self) -> float:
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self) -> int:
        v = self.c.c_ulonglong()
        if self._reasons_fn(self.h, self.c.byref(v)) != 0:
            raise RuntimeError("nvml reasons query failed")
        return int(v.value)

    def close(self):
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """Samples SM clock and clock-event (throttle) reasons every few milliseconds
    through NVML in a background thread (nvidia-smi at 100 ms as a fallback)."""

    REASONS = (("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20), ("hw_thermal_slowdown", 0x40),
               ("sw_power_cap", 0x4))

    def __init__(self, index: int, period_s: float = 0.005):
        self.index = index
        self.period = period_s
        self.samples = []  # (sm_mhz, reasons bitmask)
        self.max_mhz = None
        self._stop = threading.Event()
        self._t = None
        self._nv = None
        self.nvml_error = None

    def __enter__(self):
        try:
            self._nv = _Nvml(self.index)
            self.max_mhz = self._nv.max_sm_mhz()
            self._t = threading.Thread(target=self._poll_nvml, daemon=True)
        except Exception as e:
            self.nvml_error = repr(e)[:120]
            self._nv = None
            self._t = threading.Thread(target=self._poll_smi, daemon=True)
        self._t.start()
        return self

    def _poll_nvml(self):
        while not self._stop.is_set():
            try:
                self.samples.append((self._nv.sm_mhz(), self._nv.reasons()))
            except Exception:
                return
            self._stop.wait(self.period)

    def _poll_smi(self):
        fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={fields}",
                                     "--format=csv,noheader,nounits", "-lms", "100"],
                                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        for line in proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            try:
                mask = 0
                for (nm, bit), v in zip(self.REASONS, parts[2:6]):
                    if v.lower().startswith("active"):
                        mask |= bit
                self.samples.append((float(parts[0]), mask))
                self.max_mhz = float(parts[1])
            except (ValueError, IndexError):
                pass
            if self._stop.is_set():
                break
        proc.terminate()

    def __exit__(self, *a):
        self._stop.set()
        if self._t is not None:
            self._t.join(timeout=5)
        if self._nv is not None:
            self._nv.close()

    def summary(self):
        reasons = sorted({nm for _, m in self.samples for nm, bit in self.REASONS if m & bit})
        sm = [mhz for mhz, _ in self.samples]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "source": "nvml" if self._nv is not None else "nvidia-smi",
                **({"nvml_error": self.nvml_error} if self.nvml_error else {})}


def measured_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the
    capture was of another workload or the kernel's source changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f).get(kernel)
        if not d or d.get("workload") != workload:
            return None
        with open(os.path.join(ROOT, d["file"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        return int(d["dram_bytes"]) if sha == d["csrc_sha"] else None
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def measured_bf16_peak():
    """Dense BF16 tensor TFLOP/s for a kernel timed alone (the burst figure)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1800.0, "fallback"


# algorithmic bytes per unit of each kernel: compulsory reads and writes of one launch, plus
# 64 bytes per internal node a traversal loads (counted by an instrumented untimed run)
def kernel_bytes(name, n, m, k, nnz, nodes):
    """Algorithmic DRAM bytes of all launches of `name` in one step."""
    passes = 4  # 30-bit keys, 8-bit digits
    sort_b = lambda u: u * (12 + 16 * (passes - 1))  # first pass reads keys only, writes pairs
    table = {
        "bounds": 12 * n,
        "morton": 16 * n + 16 * m,                  # points -> codes, queries -> codes
        "onesweep_pass": sort_b(n) + sort_b(m),
        "hierarchy": 12 * n,                        # codes read, parent links written
        "fit": 52 * n + 76 * max(n - 1, 0),         # gather + leaf record, then per internal node
        "apetrei": 52 * n + 32 * max(n - 1, 0),     # perm + code + gathered point + leaf slot; node slot
        "scan": 12 * m + 8,                         # counts read twice, offsets written
        "spatial_count": 20 * m + 64 * nodes.get("spatial", 0) // 2,
        "spatial_fill": 28 * m + 4 * nnz + 64 * nodes.get("spatial", 0) // 2,
        "spatial_buffered": 20 * m + 4 * nnz + 64 * nodes.get("spatial", 0),  # one pass, rows to the buffer
        "compact": 8 * nnz + 12 * m,                                           # buffer -> CSR
        "scan_compact": 8 * nnz + 12 * m,  # counts read, offsets written, rows buffer -> CSR (one kernel)
        "nearest": m * (16 + 8 * k + 8) + 64 * nodes.get("nearest", 0),
    }
    return table.get(name)


# ---------------------------------------------------------------- GPU arm

class L2Flush:
    """Evicts L2 (126 MB) between timed steps: writes a 256 MB buffer, then reads a second
    256 MB buffer, so that the write's dirty lines go back to HBM here and not during the next
    step's first kernel."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.fill_(1.0)
        self.r.sum()


def measure_e2e(ab, args, dev, stream, flush, barrier, ws, p, q, p_h, q_h, r, k, n, m, nnz, topts, bsz, idx_buf):
    """End to end through the public API: every batch copies its points and queries from pinned
    host memory and its results (CSR rows, k-NN rows and distances) back.  Reported for a stream
    of batches (the value) and for one batch at a time."""
    import torch
    p_pin = torch.from_numpy(p_h).pin_memory()
    q_pin = torch.from_numpy(q_h).pin_memory()
    kk = min(k, n)
    outs = dict(off=torch.empty(m + 1, dtype=torch.int64).pin_memory(),
                kidx=torch.empty((m, kk), dtype=torch.int32).pin_memory(),
                kd2=torch.empty((m, kk), dtype=torch.float32).pin_memory())
    idx_pin = torch.empty(max(nnz, 1) * 2, dtype=torch.int32).pin_memory()
    pd = torch.empty_like(p)
    qd = torch.empty_like(q)

    cs = torch.cuda.Stream(device=dev)  # copy stream: overlaps transfers with the compute stream
    nnz_pin = torch.empty(1, dtype=torch.int64).pin_memory()
    ev_q = torch.cuda.Event()
    ev_sp = torch.cuda.Event()
    ev_ka = torch.cuda.Event()
    mh = m // 2

    def e2e_step():
        pd.copy_(p_pin, non_blocking=True)  # compute stream: the build needs every point
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            qd.copy_(q_pin, non_blocking=True)  # uploads while the tree builds
            ev_q.record(cs)
        bvh = ab.BVH(pd, **topts)
        stream.wait_event(ev_q)
        order = bvh.query_order(qd)
        if bsz > 0:
            off, idx = bvh.query_spatial_async(qd, r, buffer_size=bsz, order=order, indices=idx_buf)
        else:
            off, idx = bvh.query_spatial(qd, r, order=order)
        ev_sp.record(stream)
        # k-NN over the two halves of the query array (each in its own Morton order), so the
        # first half's rows download while the second half is computed
        oa, ob = bvh.query_order(qd[:mh]), bvh.query_order(qd[mh:])
        ka, da = bvh.query_nearest(qd[:mh], k, order=oa)
        ev_ka.record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(ev_sp)
            off.record_stream(cs)
            idx.record_stream(cs)
            outs["off"].copy_(off, non_blocking=True)  # downloads while the k-NN kernels run
            nnz_pin.copy_(off[-1:], non_blocking=True)
        cs.synchronize()  # the row total; the k-NN work is already queued on the compute stream
        got = int(nnz_pin[0])
        kb, db = bvh.query_nearest(qd[mh:], k, order=ob)
        with torch.cuda.stream(cs):
            idx_pin[:got].copy_(idx[:got], non_blocking=True)
            cs.wait_event(ev_ka)
            ka.record_stream(cs)
            da.record_stream(cs)
            outs["kidx"][:mh].copy_(ka, non_blocking=True)
            outs["kd2"][:mh].copy_(da, non_blocking=True)
        outs["kidx"][mh:].copy_(kb, non_blocking=True)
        outs["kd2"][mh:].copy_(db, non_blocking=True)
        stream.wait_stream(cs)  # join the copies before the end event
        bvh.destroy()
        return got

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    d2h = 0
    for _ in range(args.steps):
        flush()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        d2h = (m + 1) * 8 + got * 4 + m * kk * 8
    lat_ms = max_over_ranks(e2e_ms / args.steps, ws, dev)
    lat_value = ws * 2 * m / (lat_ms * 1e-3) / 1e6

    # A stream of independent batches, as a service runs them: batch i+1 uploads on its own copy
    # stream while batch i is computed and downloaded on a third.  Every batch still copies its
    # inputs from pinned host memory and its results back.  Three sets of device buffers rotate,
    # so an upload never waits for the compute of the batch two ahead of it (with two sets the
    # upload engine idled: 4.18 against 3.70 ms per batch; the 132 MB upload alone takes 3.67 ms
    # at the 36 GB/s the host link gives)
    NB = 3
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    pdb = [torch.empty_like(p) for _ in range(NB)]
    qdb = [torch.empty_like(q) for _ in range(NB)]
    ibuf = [torch.empty(max(nnz, 1) * 2, dtype=torch.int32, device=dev) for _ in range(NB)]
    outb = [dict(off=torch.empty(m + 1, dtype=torch.int64).pin_memory(),
                 nnz=torch.empty(1, dtype=torch.int64).pin_memory(),
                 kidx=torch.empty((m, kk), dtype=torch.int32).pin_memory(),
                 kd2=torch.empty((m, kk), dtype=torch.float32).pin_memory(),
                 idx=torch.empty(max(nnz, 1) * 2, dtype=torch.int32).pin_memory()) for _ in range(NB)]
    ev_in = [torch.cuda.Event() for _ in range(NB)]    # inputs uploaded
    ev_done = [torch.cuda.Event() for _ in range(NB)]  # computed: input buffers free again
    ev_off = [torch.cuda.Event() for _ in range(NB)]   # offsets (row total) on the host
    ev_idx = [torch.cuda.Event() for _ in range(NB)]   # rows on the host: row buffer free again
    bsz_p = bsz if bsz > 0 else 32

    def upload(i):
        b = i % NB
        with torch.cuda.stream(up):
            up.wait_event(ev_done[b])  # the batch that last read these buffers is computed
            pdb[b].copy_(p_pin, non_blocking=True)
            qdb[b].copy_(q_pin, non_blocking=True)
            ev_in[b].record(up)

    def issue(i):
        b = i % NB
        stream.wait_event(ev_in[b])
        bvh = ab.BVH(pdb[b], **topts)
        order = bvh.query_order(qdb[b])
        stream.wait_event(ev_idx[b])  # the row buffer's previous rows are on the host
        if args.queries == "concurrent":
            off, _, kidx, kd2 = bvh.query_spatial_nearest(qdb[b], r, k, buffer_size=bsz_p, order=order,
                                                          indices=ibuf[b])
        else:
            off, _ = bvh.query_spatial_async(qdb[b], r, buffer_size=bsz_p, order=order, indices=ibuf[b])
            kidx, kd2 = bvh.query_nearest(qdb[b], k, order=order)
        ev_done[b].record(stream)
        bvh.destroy()
        with torch.cuda.stream(down):
            down.wait_event(ev_done[b])
            for t in (off, kidx, kd2):
                t.record_stream(down)
            outb[b]["off"].copy_(off, non_blocking=True)
            outb[b]["nnz"].copy_(off[-1:], non_blocking=True)
            ev_off[b].record(down)
            outb[b]["kidx"].copy_(kidx, non_blocking=True)
            outb[b]["kd2"].copy_(kd2, non_blocking=True)
        return b

    def finish(b):  # the rows of batch b once its total is on the host
        ev_off[b].synchronize()
        got = int(outb[b]["nnz"][0])
        with torch.cuda.stream(down):
            outb[b]["idx"][:got].copy_(ibuf[b][:got], non_blocking=True)
            ev_idx[b].record(down)
        return got

    def stream_batches(count):
        prev, got = None, 0
        upload(0)
        for i in range(count):
            if i + 1 < count:
                upload(i + 1)  # queued at once: the copy engine starts as soon as its buffers are free
            b = issue(i)
            if prev is not None:
                got += finish(prev)
            prev = b
        return got + finish(prev)

    stream_batches(max(1, args.warmup))
    torch.cuda.synchronize()
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(up)
    got_all = stream_batches(args.steps)
    stream.wait_stream(up)
    stream.wait_stream(down)
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, ws, dev)
    e2e_value = ws * 2 * m / (e2e_ms * 1e-3) / 1e6
    d2h = (m + 1) * 8 + got_all // args.steps * 4 + m * kk * 8

    e2e = {"value": round(e2e_value, 3), "unit": UNIT, "ms_per_step": round(e2e_ms, 4),
           "h2d_bytes_per_step": int(p_h.nbytes + q_h.nbytes), "d2h_bytes_per_step": int(d2h),
           "pipelined": f"{args.steps} batches in one timed region: batch i+1 uploads while batch i is "
                        "computed and downloaded (three streams, three buffer sets)",
           "single_batch": {"value": round(lat_value, 3), "ms_per_step": round(lat_ms, 4),
                            "overlap": "queries upload during the build, spatial rows download during the "
                                       "k-NN query, k-NN in two halves with the first half's rows "
                                       "downloading during the second"}}
    return e2e


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1908_11807_b300 as ab

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_name, n, m, k = WORKLOADS[args.workload]
    seed = datagen.SEED0 + 2
    p_h, q_h = datagen.workload(dist_name, n, m, seed)
    r = datagen.radius_for_mean(n, dist_name)
    p = torch.from_numpy(p_h).to(dev)
    q = torch.from_numpy(q_h).to(dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    # launch parameters from the autotuner, tuned on another draw of the same distribution
    tuned = {"block_size": 0, "stack_smem": 0, "buffer_size": 0}
    if args.launch:
        fields = [int(x) for x in args.launch.split(",")]
        tuned = {"block_size": fields[0], "stack_smem": fields[1], "buffer_size": fields[2], "source": "--launch"}
        if len(fields) > 3:
            tuned["knn_anchor"] = fields[3]
    elif not args.no_tune:
        from paper_1908_11807_b300 import autotune
        # a full-size draw: the walk form of the tree bound ranks differently at lower query density
        tp, tq = datagen.workload(dist_name, n, m, seed + 1000)
        tuned = autotune.tune(torch.from_numpy(tp).to(dev), torch.from_numpy(tq).to(dev), r, k, dist_name)
        del tp, tq
    # validate=0: the build runs without a host round trip; non-finite input is reported by
    # arborx_check, which runs after every step outside the timed interval
    topts = {"block_size": tuned["block_size"], "stack_smem": tuned["stack_smem"], "validate": 0,
             "knn_anchor": int(tuned.get("knn_anchor") or 3)}
    bsz = int(tuned["buffer_size"] or 0)

    # one-pass spatial rows go straight into a preallocated buffer (no host round trip inside the
    # step); its capacity, m * max(bsz, 32), is three times the mean-10 result count
    idx_buf = torch.empty(m * max(bsz, 32), dtype=torch.int32, device=dev) if bsz > 0 else None

    concurrent = bsz > 0 and args.queries == "concurrent"

    def step(points, queries, conc=None, **opts):
        conc = concurrent if conc is None else conc
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        bvh = ab.BVH(points, **topts, **opts)
        ev[1].record(stream)
        order = bvh.query_order(queries)
        if conc:
            # one call: the nearest traversal on the handle's second stream, overlapping the
            # spatial query's compaction and overflow pass; both joined back into `stream`
            off, idx, kidx, kd2 = bvh.query_spatial_nearest(queries, r, k, buffer_size=bsz, order=order,
                                                            indices=idx_buf)
            ev[2].record(stream)
            ev[3].record(stream)
            return ev, (off, idx, kidx, kd2), bvh
        if bsz > 0:
            off, idx = bvh.query_spatial_async(queries, r, buffer_size=bsz, order=order, indices=idx_buf)
        else:
            off, idx = bvh.query_spatial(queries, r, order=order)
        ev[2].record(stream)
        kidx, kd2 = bvh.query_nearest(queries, k, order=order)
        ev[3].record(stream)
        return ev, (off, idx, kidx, kd2), bvh

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(p, q)[2].destroy()
    barrier()

    # internal nodes loaded per query (instrumented, untimed run)
    _, _, sbvh = step(p, q, stats=1)
    st = sbvh.stats()
    sbvh.destroy()
    nodes = {"spatial": int(st["spatial_nodes"]), "nearest": int(st["nearest_nodes"])}

    ab.profile_enable(True)
    ab.profile_report()  # reset
    phase = np.zeros(3)
    total_ms = 0.0
    nnz = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush()  # evict L2 between steps (outside the timed interval)
            barrier()
            ev, res, bvh = step(p, q)
            torch.cuda.synchronize()
            bvh.check()
            bvh.destroy()
            t = [ev[0].elapsed_time(e) for e in ev[1:]]
            phase += np.array([t[0], t[1] - t[0], t[2] - t[1]])
            total_ms += t[2]
            nnz = int(res[0][-1].item())
    prof = ab.profile_report()
    launches = int(sum(c for c, _ in prof.values()))  # every launch of the K timed steps
    prof_overlapped = prof
    seq_phase = None
    if concurrent:
        # Per-kernel times for the kernel table and the roofline come from the same number of
        # steps run one kernel after another (the two traversals of the step above share the
        # GPU, so each one's event interval also holds the other's work)
        seq_phase = np.zeros(3)
        for _ in range(args.steps):
            flush()
            barrier()
            ev, _, bvh = step(p, q, conc=False)
            torch.cuda.synchronize()
            bvh.check()
            bvh.destroy()
            t = [ev[0].elapsed_time(e) for e in ev[1:]]
            seq_phase += np.array([t[0], t[1] - t[0], t[2] - t[1]])
        seq_phase /= args.steps
        prof = ab.profile_report()
    ab.profile_enable(False)
    clocks = clk.summary()

    step_ms = max_over_ranks(total_ms / args.steps, ws, dev)
    value = ws * 2 * m / (step_ms * 1e-3) / 1e6
    build_ms, spatial_ms, knn_ms = phase / args.steps

    # ---- end to end: pinned host buffers in, results back to host, every step
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(ab, args, dev, stream, flush, barrier, ws, p, q, p_h, q_h, r, k, n, m, nnz, topts, bsz,
                          idx_buf)

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    kernels = {}
    dom = None
    for name, (cnt, ms) in prof.items():
        per_step_ms = ms / args.steps
        kernels[name] = {"launches_per_step": cnt / args.steps, "ms_per_step": round(per_step_ms, 4)}
        if dom is None or ms > prof[dom][1]:
            dom = name
    tot_k = sum(ms for _, ms in prof.values())
    for name in kernels:
        kernels[name]["share"] = round(prof[name][1] / tot_k, 4) if tot_k else None
    roofline = None
    if dom is not None:
        b = kernel_bytes(dom, n, m, k, nnz, nodes)
        dom_ms = prof[dom][1] / args.steps
        if b is not None and dom_ms > 0:
            achieved = b / (dom_ms * 1e-3) / 1e9
            traffic = measured_traffic(dom, args.workload) if prof[dom][0] == args.steps else None
            traversal = dom in ("nearest", "spatial_buffered", "spatial_count", "spatial_fill")
            roofline = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1),
                        "peak": peak, "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                        "traffic": traffic, "algorithmic_bytes_per_step": int(b)}
            if traversal:
                # the axis is HBM bandwidth, but achieved counts every 64-byte node the traversal loads
                # (a node-fetch rate, mostly served by L2); what limits the kernel is node-load latency
                # and its divergent instruction stream, and what HBM itself delivered is the measured
                # DRAM traffic over the same time
                roofline["limiter"] = ("node-load latency and divergent instruction issue (not HBM): "
                                       "achieved is a node-fetch rate, mostly from L2")
                if traffic:
                    dram = traffic / (dom_ms * 1e-3) / 1e9
                    roofline["dram_achieved"] = round(dram, 1)
                    roofline["dram_frac"] = round(dram / peak, 4)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: n={n} {dist_name} points, m={m} same-distribution queries, "
                               f"radius {r:.7g} (mean 10 neighbours), k={k}",
                   "n": n, "m": m, "k": k, "radius": r, "key_bits": 30, "parallelism": f"replicas{ws}",
                   "build_validate": "asynchronous (arborx_check after each step, untimed)",
                   "l2": "flushed between steps (256 MB write, then a 256 MB read of a second buffer)"},
        "components": ({"build_mpts_s": round(n / (build_ms * 1e-3) / 1e6, 2),
                        "queries_mq_s": round(2 * m / (spatial_ms * 1e-3) / 1e6, 2),
                        "build_ms": round(build_ms, 4),
                        "queries_ms": round(spatial_ms, 4), "nnz": nnz,
                        "queries": "query order, then the radius and k-NN queries in one call "
                                   "(arborx_query_spatial_nearest: the k-NN traversal on a second stream)",
                        "sequential_pass": {"note": "the same steps with the two queries one after the "
                                                    "other (the pass that times the kernels)",
                                            "build_ms": round(float(seq_phase[0]), 4),
                                            "radius_ms": round(float(seq_phase[1]), 4),
                                            "knn_ms": round(float(seq_phase[2]), 4),
                                            "step_ms": round(float(seq_phase.sum()), 4)}}
                       if concurrent else
                       {"build_mpts_s": round(n / (build_ms * 1e-3) / 1e6, 2),
                        "radius_mq_s": round(m / (spatial_ms * 1e-3) / 1e6, 2),
                        "knn_mq_s": round(m / (knn_ms * 1e-3) / 1e6, 2),
                        "build_ms": round(build_ms, 4), "radius_ms": round(spatial_ms, 4),
                        "knn_ms": round(knn_ms, 4), "nnz": nnz}),
        "kernels": kernels,
        "kernels_source": ("a second pass of the same number of steps with the radius and k-NN queries one "
                           "after the other on one stream: in the timed step the two traversals overlap, so "
                           "each one's event interval holds part of the other's work (kernels_overlapped)"
                           if concurrent else "the timed steps"),
        "kernels_overlapped": ({name: round(ms / args.steps, 4) for name, (cnt, ms) in prof_overlapped.items()}
                               if concurrent else None),
        "tuned": tuned,
        "traversal": {"spatial_nodes_per_query": round(nodes["spatial"] / m, 2),
                      "nearest_nodes_per_query": round(nodes["nearest"] / m, 2), "node_bytes": 64},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": launches,
        "gpu_launches_per_step": round(launches / args.steps, 2),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        extras = set(args.extras.split(","))
        if "query_ordering" in extras:
            line["query_ordering"] = ordering_extra(ab, p, q, r, k, topts)
        if "learned" in extras:
            line["learned"] = learned_extra(ab, dev)
        if "mlp" in extras:
            line["mlp"] = mlp_extra(ab, dev)
        if "batched" in extras:
            line["batched"] = batched_extra(ab, dev)
        if "intersects" in extras:
            line["intersects"] = intersects_extra(ab, dev, topts)
        if "configs" in extras:
            line["configs"] = configs_extra(ab, dev, topts)
        if "cpu_configs" in extras and not args.no_cpu_baseline:
            line["cpu_configs"] = cpu_configs_extra()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, p_h, q_h, r, k, n, m, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _time_ms(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def ordering_extra(ab, p, q, r, k, topts):
    """Query ordering (Sec. 2.2.3): the same queries traversed in Morton order (the query sort
    included in the time) and in input order, with the internal nodes loaded per query."""
    out = {}
    for name, sq in (("sorted", 1), ("unsorted", 0)):
        bvh = ab.BVH(p, sort_queries=sq, **topts)
        knn_ms = _time_ms(lambda: bvh.query_nearest(q, k))
        sp_ms = _time_ms(lambda: bvh.query_spatial(q, r))
        bvh.destroy()
        bvh = ab.BVH(p, sort_queries=sq, stats=1, **topts)  # node counts (instrumented, not timed)
        bvh.stats()
        bvh.query_nearest(q, k)
        nodes = bvh.stats()["nearest_nodes"] / q.shape[0]
        out[name] = {"knn_ms": round(knn_ms, 3), "spatial_2p_ms": round(sp_ms, 3),
                     "knn_nodes_per_query": round(nodes, 1)}
        bvh.destroy()
    out["knn_speedup_from_ordering"] = round(out["unsorted"]["knn_ms"] / out["sorted"]["knn_ms"], 2)
    out["spatial_speedup_from_ordering"] = round(out["unsorted"]["spatial_2p_ms"] / out["sorted"]["spatial_2p_ms"], 2)
    return out


def intersects_extra(ab, dev, topts):
    """Box-intersection queries over the 1e7-box tree (centres uniform in the unit cube, half-widths
    uniform in [0, 1e-3]): 1e6 cube queries with the half-width that meets 10 boxes on average.
    The query time includes the Morton order of the query boxes; rows go to a caller buffer."""
    import torch
    n, m = 10_000_000, 1_000_000
    seed = datagen.SEED0 + 2
    half = datagen.box_half_for_mean(n)
    b = torch.from_numpy(datagen.boxes(n, seed)).to(dev)
    qb = torch.from_numpy(datagen.query_cubes(m, seed, half)).to(dev)
    idx = torch.empty(m * 32, dtype=torch.int32, device=dev)
    build_ms = _time_ms(lambda: ab.BVH(b, **topts).destroy())
    bvh = ab.BVH(b, **topts)

    def query(t):
        order = t.query_order_boxes(qb)
        return t.query_intersects_async(qb, buffer_size=32, order=order, indices=idx)

    query_ms = _time_ms(lambda: query(bvh))
    off, _ = query(bvh)
    bvh.check()
    nnz = int(off[-1].item())
    bvh.destroy()
    sbvh = ab.BVH(b, stats=1, **topts)  # node counts from an instrumented tree (its atomics are not timed)
    sbvh.stats()
    query(sbvh)
    nodes = sbvh.stats()["spatial_nodes"] / m
    sbvh.destroy()
    node_bytes = 24 * m + 4 * nnz + 64 * nodes * m
    return {"workload": f"1e7 boxes (half-widths U[0,1e-3]), 1e6 cube queries of half-width {half:.4g}",
            "build_ms": round(build_ms, 3), "build_mboxes_s": round(n / (build_ms * 1e-3) / 1e6, 1),
            "query_ms": round(query_ms, 3), "query_mq_s": round(m / (query_ms * 1e-3) / 1e6, 1),
            "hits_per_query": round(nnz / m, 2), "nodes_per_query": round(nodes, 2),
            "node_fetch_gbs": round(node_bytes / (query_ms * 1e-3) / 1e9, 1)}


def configs_extra(ab, dev, topts):
    """Each test configuration's shape timed like the headline step (build, Morton order of the
    queries, radius query in the scheme the tuner picks for that radius, k-NN), device-resident
    inputs, best of three: the small cube,
    the paper-scale cube and hollow sphere at 1e6 and 1e7 points, the 1e7-box build, and the
    256^3 lattice with 1e6 query sites at r = 1, 2.5, 4 and k = 27."""
    import torch
    from paper_1908_11807_b300 import autotune
    seed = datagen.SEED0 + 2
    out = {}

    def run(name, p_h, q_h, radii, k):
        p = torch.from_numpy(p_h).to(dev)
        q = torch.from_numpy(q_h).to(dev)
        build_ms = _time_ms(lambda: ab.BVH(p, **topts).destroy())
        # the queried tree keeps its sorted leaf order, so that the per-radius pick can also choose
        # the traversal that takes wholly contained subtrees from it
        bvh = ab.BVH(p, keep_order=1, **topts)
        order = bvh.query_order(q)
        order_ms = _time_ms(lambda: bvh.query_order(q))
        row = {"n": int(p_h.shape[0]), "m": int(q_h.shape[0]), "build_ms": round(build_ms, 3),
               "build_mpts_s": round(p_h.shape[0] / build_ms / 1e3, 1), "order_ms": round(order_ms, 3)}
        for r in radii:
            # the row-buffer width for this radius (0: two passes), from its hit-count distribution
            pick = autotune.pick_buffer(bvh, q, r, order=order)
            bs = pick["buffer_size"]
            off, _ = bvh.query_spatial(q, r, order=order, buffer_size=bs)  # sizes the result buffer
            nnz = int(off[-1].item())
            rows = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
            if bs > 0:
                sp_ms = _time_ms(lambda: bvh.query_spatial_async(q, r, buffer_size=bs, order=order, indices=rows))
            else:
                sp_ms = _time_ms(lambda: bvh.query_spatial(q, r, order=order))
            bvh.check()
            row[f"radius_{r:.4g}"] = {"ms": round(sp_ms, 3), "mq_s": round(q_h.shape[0] / sp_ms / 1e3, 1),
                                      "hits_per_query": round(nnz / q_h.shape[0], 2), "buffer_size": bs,
                                      "buffer_candidates_ms": pick["ms"], "emit_subtrees": pick["emit_subtrees"],
                                      "emit_ms": pick.get("emit_ms")}
            bvh.emit_subtrees(False)
            del rows
        if k:
            kn_ms = _time_ms(lambda: bvh.query_nearest(q, k, order=order))
            row[f"knn_{k}"] = {"ms": round(kn_ms, 3), "mq_s": round(q_h.shape[0] / kn_ms / 1e3, 1)}
        bvh.destroy()
        out[name] = row

    for dist in ("cube", "hollow_sphere"):
        for n in (1_000_000, 10_000_000):
            p_h, q_h = datagen.workload(dist, n, 1_000_000, seed)
            run(f"{dist}_{n:.0e}".replace("+0", ""), p_h, q_h, [datagen.radius_for_mean(n, dist)], 10)
    p_h, q_h = datagen.workload("cube", 10_000, 10_000, seed)
    run("cube_1e4", p_h, q_h, [datagen.radius_for_mean(10_000, "cube")], 10)
    b = torch.from_numpy(datagen.boxes(10_000_000, seed)).to(dev)
    bms = _time_ms(lambda: ab.BVH(b, **topts).destroy())
    out["boxes_1e7"] = {"n": 10_000_000, "build_ms": round(bms, 3), "build_mboxes_s": round(1e7 / bms / 1e3, 1)}
    del b
    _, sites = datagen.lattice_sites(1_000_000, datagen.SEED0 + 3)
    run("lattice_256", datagen.lattice(), sites, [1.0, 2.5, 4.0], 27)
    return out


def cpu_configs_extra(sample=100_000):
    """The oracle on the host cores at each test configuration's shape: its CPU BVH (median
    split, leaf 4, OpenMP) built over all n points and queried with the first `sample` queries
    (radius for a mean of 10 neighbours, k = 10; the lattice at r = 1, 2.5, 4 and k = 27), and
    brute force at the small cube.  Rates are of what was timed: build Mpts/s over all n, query
    Mq/s over the sampled queries."""
    import oracle
    seed = datagen.SEED0 + 2
    out = {"cores": oracle.threads(), "queries_timed": sample}

    def run(name, p_h, q_h, radii, k, brute=False):
        qs = q_h[:sample]
        t0 = time.perf_counter()
        tree = oracle.CpuBVH(p_h)
        t1 = time.perf_counter()
        row = {"n": int(p_h.shape[0]), "build_s": round(t1 - t0, 3),
               "build_mpts_s": round(p_h.shape[0] / (t1 - t0) / 1e6, 2)}
        for r in radii:
            t0 = time.perf_counter()
            off, _ = tree.spatial(qs, r)
            dt = time.perf_counter() - t0
            row[f"radius_{r:.4g}"] = {"mq_s": round(len(qs) / dt / 1e6, 4), "s": round(dt, 3),
                                      "hits_per_query": round(float(off[-1]) / len(qs), 2)}
        t0 = time.perf_counter()
        tree.nearest(qs, k)
        dt = time.perf_counter() - t0
        row[f"knn_{k}"] = {"mq_s": round(len(qs) / dt / 1e6, 4), "s": round(dt, 3)}
        del tree
        if brute:
            t0 = time.perf_counter()
            oracle.spatial_brute(p_h, qs, radii[0])
            dt_s = time.perf_counter() - t0
            t0 = time.perf_counter()
            oracle.nearest_brute(p_h, qs, k)
            dt_k = time.perf_counter() - t0
            row["brute_force"] = {"radius_mq_s": round(len(qs) / dt_s / 1e6, 4),
                                  f"knn_{k}_mq_s": round(len(qs) / dt_k / 1e6, 4)}
        out[name] = row

    p_h, q_h = datagen.workload("cube", 10_000, 10_000, seed)
    run("cube_1e4", p_h, q_h, [datagen.radius_for_mean(10_000, "cube")], 10, brute=True)
    for dist in ("cube", "hollow_sphere"):
        for n in (1_000_000, 10_000_000):
            p_h, q_h = datagen.workload(dist, n, sample, seed)
            run(f"{dist}_{n:.0e}".replace("+0", ""), p_h, q_h, [datagen.radius_for_mean(n, dist)], 10)
    b = datagen.boxes(10_000_000, seed)
    t0 = time.perf_counter()
    tree = oracle.CpuBVH(b)
    dt = time.perf_counter() - t0
    del tree
    out["boxes_1e7"] = {"n": 10_000_000, "build_s": round(dt, 3), "build_mboxes_s": round(1e7 / dt / 1e6, 2)}
    del b
    _, sites = datagen.lattice_sites(sample, datagen.SEED0 + 3)
    run("lattice_256", datagen.lattice(), sites, [1.0, 2.5, 4.0], 27)
    return out


def learned_extra(ab, dev):
    """Learned initial bound vs plain nearest traversal: 1e7 points and 1e7 queries from a
    64-Gaussian mixture, regressor trained on 1e6 exact labels by the library's kernels."""
    import torch
    from paper_1908_11807_b300 import autotune
    n, m, mt = 10_000_000, 10_000_000, 1_000_000
    seed = datagen.SEED0 + 5
    p = torch.from_numpy(datagen.gaussian_mixture(n, seed)).to(dev)
    q = torch.from_numpy(datagen.gaussian_mixture(m, seed, datagen.STREAM_QUERIES)).to(dev)
    qt = torch.from_numpy(datagen.gaussian_mixture(mt, seed, datagen.STREAM_TRAIN)).to(dev)
    q_tune = torch.from_numpy(datagen.gaussian_mixture(m, seed, datagen.STREAM_HELDOUT)).to(dev)
    out = {"workload": "gaussian mixture (64 components), n=1e7 points, m=1e7 queries, 1e6 training labels",
           "plain": "the library's default nearest query: its traversal starts from the tree's own bound "
                    "(knn_anchor = 3: gathered on the first descent for k up to 10, the walk through the "
                    "child holding the query for wider lists); also timed: the paper's unbounded start "
                    "(knn_anchor = 0), the far-corner walk (1) and the query-path walk (2)",
           "margin_tuned_on": "a held-out draw of 1e7 queries from the same mixture (not the timed set)",
           "unit": "ms per query batch"}
    bvh = ab.BVH(p)
    bvh_paper = ab.BVH(p, knn_anchor=0)
    bvh_far = ab.BVH(p, knn_anchor=1)
    bvh_path = ab.BVH(p, knn_anchor=2)
    order = bvh.query_order(q)
    for k in (10, 50):
        g = np.random.default_rng(seed)
        init = np.concatenate([g.standard_normal(192) * np.sqrt(2 / 3), np.zeros(64),
                               g.standard_normal(4096) * np.sqrt(2 / 64), np.zeros(64),
                               g.standard_normal(64) * np.sqrt(1 / 64), np.zeros(1)]).astype(np.float32)
        params = torch.from_numpy(init).to(dev)
        t0 = time.perf_counter()
        loss = bvh.mlp_train(params, qt, k, epochs=1200, batch=2048, lr=5e-3, lr_final=1e-5)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        # the margin is tuned on a held-out draw of 1e7 queries from the same mixture (full size, so
        # that the Morton neighbours of the second pass are as dense as in the timed set)
        margin = autotune.tune_margin(bvh, q_tune, k, params)
        plain_ms = _time_ms(lambda: bvh.query_nearest(q, k, order=order))
        learned_ms = _time_ms(lambda: bvh.query_nearest_learned(q, k, params, margin, order=order))
        pi, pd = bvh.query_nearest(q, k, order=order)
        li, ld, fb = bvh.query_nearest_learned(q, k, params, margin, order=order, count_fallbacks=True)
        same = bool(torch.equal(pi, li) and torch.equal(pd, ld))
        # what a perfect regressor could give: the exact k-th distance (plus 2^-10) as the bound
        b2 = (pd[:, -1] * (1 + 2 ** -10)).contiguous()
        exact_ms = _time_ms(lambda: bvh.query_nearest_bounded(q, k, b2, order=order))
        del b2
        # the paper's traversal as published: no initial bound at all (knn_anchor = 0); and the tree
        # bound's walk forms (knn_anchor = 1, the far-corner walk; 2, the query-path walk)
        paper_ms = _time_ms(lambda: bvh_paper.query_nearest(q, k, order=order))
        far_ms = _time_ms(lambda: bvh_far.query_nearest(q, k, order=order))
        path_ms = _time_ms(lambda: bvh_path.query_nearest(q, k, order=order))
        out[f"k{k}"] = {"plain_ms": round(plain_ms, 3), "learned_ms": round(learned_ms, 3),
                        "speedup": round(plain_ms / learned_ms, 3), "identical_results": same,
                        "plain_mq_s": round(m / plain_ms / 1e3, 1), "learned_mq_s": round(m / learned_ms / 1e3, 1),
                        "margin": margin, "fallback_fraction": round(fb / m, 4),
                        "train_s": round(train_s, 2), "final_loss": round(float(loss[-1].item()), 4),
                        "exact_bound_ms": round(exact_ms, 3), "exact_bound_speedup": round(plain_ms / exact_ms, 3),
                        "unbounded_start_ms": round(paper_ms, 3),
                        "learned_speedup_over_unbounded_start": round(paper_ms / learned_ms, 3),
                        "far_corner_tree_bound_ms": round(far_ms, 3),
                        "learned_speedup_over_far_corner_tree_bound": round(far_ms / learned_ms, 3),
                        "query_path_tree_bound_ms": round(path_ms, 3),
                        "learned_speedup_over_query_path_tree_bound": round(path_ms / learned_ms, 3)}
        del pi, pd, li, ld
    del q_tune
    bvh.destroy()
    bvh_paper.destroy()
    bvh_far.destroy()
    bvh_path.destroy()
    return out


def mlp_extra(ab, dev):
    """Bound-regressor inference (3 -> 64 -> 64 -> 1) over 1e7 queries: the BF16 tcgen05 kernel
    (the 64 x 64 layer on the tensor cores, accumulators in tensor memory) against the FP32
    CUDA-core form, with the flop and byte rates of the tensor-core launch."""
    import torch
    n, m = 1_000_000, 10_000_000
    seed = datagen.SEED0 + 5
    p = torch.from_numpy(datagen.gaussian_mixture(n, seed)).to(dev)
    q = torch.from_numpy(datagen.gaussian_mixture(m, seed, datagen.STREAM_QUERIES)).to(dev)
    g = np.random.default_rng(seed)
    init = np.concatenate([g.standard_normal(192) * np.sqrt(2 / 3), np.zeros(64),
                           g.standard_normal(4096) * np.sqrt(2 / 64), np.zeros(64),
                           g.standard_normal(64) * np.sqrt(1 / 64), np.zeros(1)]).astype(np.float32)
    params = torch.from_numpy(init).to(dev)
    bvh = ab.BVH(p)
    tc_ms = _time_ms(lambda: bvh.mlp_forward(params, q, tensor_cores=True), reps=5)
    fp32_ms = _time_ms(lambda: bvh.mlp_forward(params, q, tensor_cores=False), reps=5)
    bvh.destroy()
    hbm, hbm_kind = measured_peaks()
    bf16, bf16_kind = measured_bf16_peak()
    flop = 2 * (3 * 64 + 64 * 64 + 64) * m    # every layer
    tensor_flop = 2 * 64 * 64 * m             # the layer on the tensor cores
    nbytes = (12 + 4) * m                     # query in, output out
    return {"workload": f"gaussian mixture queries, m={m}, random-init regressor (4481 parameters)",
            "tensor_core_ms": round(tc_ms, 4), "fp32_ms": round(fp32_ms, 4),
            "speedup_over_fp32": round(fp32_ms / tc_ms, 2),
            "tflops_all_layers": round(flop / tc_ms / 1e9, 1),
            "tensor_layer_frac_of_bf16_peak": round(tensor_flop / tc_ms / 1e9 / bf16, 4),
            "hbm_gbs": round(nbytes / tc_ms / 1e6, 1),
            "hbm_frac": round(nbytes / tc_ms / 1e6 / hbm, 4),
            "peak_source": f"bf16 {bf16_kind}, hbm {hbm_kind}"}


def batched_extra(ab, dev):
    """512 independent clouds (sizes log-uniform in [1e3, 1e5], cube or hollow sphere, k in
    {1, 10, 32}): one graph-replayed batch vs a per-cloud build + query loop."""
    import torch
    w = datagen.batched_workload(512, datagen.SEED0 + 4)
    pts = [c["points"] for c in w]
    qs = [c["queries"] for c in w]
    ks = np.array([c["k"] for c in w], np.int32)
    po = np.concatenate([[0], np.cumsum([len(x) for x in pts])]).astype(np.int64)
    qo = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
    P = torch.from_numpy(np.concatenate(pts)).to(dev)
    Q = torch.from_numpy(np.concatenate(qs)).to(dev)
    from paper_1908_11807_b300 import autotune
    b0 = ab.Batch(po, qo, ks)  # library defaults
    o0 = b0.run(P, Q, use_graph=True)
    default_ms = _time_ms(lambda: b0.run(P, Q, use_graph=True, out=(o0[0], o0[1], o0[2])), reps=5)
    tuned = autotune.tune_batch(po, qo, ks, P, Q)
    b = ab.Batch(po, qo, ks, block_size=tuned["block_size"], stack_smem=tuned["stack_smem"],
                 queries_per_warp=tuned["queries_per_warp"], knn_heap_from=tuned["knn_heap_from"],
                 knn_anchor=tuned["knn_anchor"])
    out_bufs = b.run(P, Q, use_graph=True)
    graph_ms = _time_ms(lambda: b.run(P, Q, use_graph=True, out=(out_bufs[0], out_bufs[1], out_bufs[2])), reps=5)
    same = bool(torch.equal(o0[1], out_bufs[1]) and torch.equal(o0[2], out_bufs[2]))
    del o0
    b0.destroy()
    eager_ms = _time_ms(lambda: b.run(P, Q, use_graph=False), reps=3)
    # per-kernel device time of one eager run (the profiler's event pairs cannot sit in a graph)
    ab.profile_enable(True)
    ab.profile_report()
    b.run(P, Q, use_graph=False)
    torch.cuda.synchronize()
    per_kernel = {k_: round(ms_, 3) for k_, (_, ms_) in sorted(ab.profile_report().items(), key=lambda x: -x[1][1])}
    ab.profile_enable(False)
    b.check()
    pd = [P[po[c]:po[c + 1]] for c in range(512)]
    qd = [Q[qo[c]:qo[c + 1]] for c in range(512)]

    def loop():
        for c in range(512):
            t = ab.BVH(pd[c], validate=0)
            t.query_nearest(qd[c], int(ks[c]))
            t.destroy()
    loop_ms = _time_ms(loop, reps=2)
    mtot = int(qo[-1])
    b.destroy()
    return {"workload": f"512 clouds, {int(po[-1])} points, {mtot} queries, k in {{1,10,32}}",
            "tuned": tuned, "default_tiles_graph_ms": round(default_ms, 3), "tuned_equals_default": same,
            "per_kernel_ms": per_kernel,
            "graph_ms": round(graph_ms, 3), "eager_batch_ms": round(eager_ms, 3), "per_cloud_loop_ms": round(loop_ms, 3),
            "graph_mq_s": round(mtot / graph_ms / 1e3, 1), "loop_mq_s": round(mtot / loop_ms / 1e3, 1),
            "speedup_vs_loop": round(loop_ms / graph_ms, 2)}


# ---------------------------------------------------------------- CPU oracle arm

def cpu_step(p_h, q_h, r, k, sample):
    """One measured step of the CPU oracle: its BVH built over all points, then ``sample`` radius
    and ``sample`` k-nearest queries.  Returns the seconds of (whole step, build, radius, nearest);
    nothing is extrapolated."""
    import oracle
    t0 = time.perf_counter()
    tree = oracle.CpuBVH(p_h)
    t1 = time.perf_counter()
    qs = q_h[:sample]
    tree.spatial(qs, r)
    t2 = time.perf_counter()
    tree.nearest(qs, k)
    t3 = time.perf_counter()
    del tree
    return t3 - t0, t1 - t0, t2 - t1, t3 - t2


def cpu_baseline(args, p_h, q_h, r, k, n, m, budget_s=20.0):
    """The oracle's CPU BVH on the host cores over the whole workload (all n points, all m
    queries), as measured: a few steps within about ``budget_s`` seconds, median reported."""
    import oracle
    cores = oracle.threads()
    steps = []
    t_start = time.perf_counter()
    while True:
        steps.append(cpu_step(p_h, q_h, r, k, m))
        if time.perf_counter() - t_start > budget_s * 0.5 or len(steps) >= 3:
            break
    med = sorted(steps)[len(steps) // 2]
    return {"value": round(2 * m / med[0] / 1e6, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole workload, measured: CPU BVH (median split, leaf 4, OpenMP) built over all {n} "
                      f"points, then all {m} radius and all {m} k={k} queries; median of {len(steps)} steps",
            "step_s": round(med[0], 3), "build_s": round(med[1], 3), "spatial_s": round(med[2], 4),
            "knn_s": round(med[3], 4)}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    dist_name, n, m, k = WORKLOADS[args.workload]
    seed = datagen.SEED0 + 2
    p_h, q_h = datagen.workload(dist_name, n, m, seed)
    r = datagen.radius_for_mean(n, dist_name)
    sample = m if args.ref_queries is None else max(1, min(m, args.ref_queries))
    for _ in range(args.warmup):
        cpu_step(p_h, q_h, r, k, sample)
    times = [cpu_step(p_h, q_h, r, k, sample)[0] for _ in range(args.steps)]
    step_s = float(np.mean(times))
    value = 2 * sample / step_s / 1e6
    cores = oracle.threads()
    what = (f"per step, measured: CPU BVH built over all {n} points, then {sample} radius + {sample} k={k} "
            f"queries ({'all' if sample == m else 'the first'} of the workload's {m})")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: n={n} {dist_name} points, m={m} same-distribution queries, "
                               f"radius {r:.7g} (mean 10 neighbours), k={k}", "n": n, "m": m, "k": k,
                   "queries_timed_per_step": sample},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": what},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="cube_1e7", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-queries", type=int, default=None,
                    help="reference arm: queries of each kind timed per step (default: all m)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the learned-bound and batched measurements")
    ap.add_argument("--extras", default="query_ordering,learned,mlp,batched,intersects,configs,cpu_configs",
                    help="comma-separated extra measurements to run (after the headline step)")
    ap.add_argument("--no-tune", action="store_true", help="default launch parameters instead of the autotuner's")
    ap.add_argument("--queries", default="concurrent", choices=["concurrent", "sequential"],
                    help="radius and k-NN queries of a step in one call on two streams (arborx_query_spatial_nearest) "
                         "or one after the other on one stream")
    ap.add_argument("--launch", default=None,
                    help="block,stack,buffer[,knn_anchor]: fixed traversal launch parameters (skips the autotuner)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "b300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
