#!/usr/bin/env python
"""Benchmark of the GB300 3-way hash join: input tuples/s of the linear
friends-of-friends-of-friends self-join F |x| F |x| F (COUNT(*) GROUP BY A)
on a synthetic power-law graph of 2^20 vertices (Zipf s=1.1 degrees capped at
4096, mean degree 32, ~3.3e7 directed edges), multiway vs cascade, exact
counts.

Prints one JSON line.  `python bench.py --gpus N --steps K --warmup W`; under
torchrun every rank runs its own replica of the workload (the join is one
problem per GPU; replicas only) and rank 0 reports the aggregate.  With one
GPU the line also carries the other workloads (sub-objects): the uniform
linear join of 2^16 tuples per relation, the triangle join on a 2^22-vertex
graph (count, GROUP BY A, materialised list, chunked cascade), the batch of
4096 queries replayed from a CUDA graph, the headline graph with its rows
shuffled, and the star, skewed, four-relation and Flajolet-Martin variants.
Exactness flags compare with the CPU oracle; every oracle call sits in the
cpu_baseline_* functions.

--impl reference times the CPU oracle (single-threaded C hash join) on the
same workload and metric.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3-way join input tuples/s + % HBM roofline, multiway vs cascade, exact counts"
UNIT = "tuples/s"
L2_NOTE = "every input column pair (262 MB) exceeds the 129 MB L2; no flush"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel from
# one ncu capture, per step of the benchmark workload, valid while the sources
# the kernel is built from are unchanged (digest of those files).  The
# captures ran on the 2^19-vertex graph (16,090,397 edges) and are scaled by
# the edge count to the 2^20-vertex graph (32,804,288 edges, x 2.0387): the
# traffic grows with the tuples streamed and the tables double with the
# vertex count as well.
TRAFFIC = {
    "part_scatter": {"bytes_per_step": 970_700_000, "digest": "a8955b800db65c70",
                     "sources": ["csrc/partition.cu", "csrc/common.cuh", "csrc/internal.h", "csrc/skew.h"]},
    "w_build": {"bytes_per_step": 282_970_000, "digest": "31653c3bfe715b04",
                "sources": ["csrc/linear_l2.cu", "csrc/linear_l2.h", "csrc/common.cuh", "csrc/internal.h",
                            "csrc/skew.h", "csrc/tables.h", "csrc/warp_runs.cuh"]},
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
def summarize_clocks(lines, t0=None, t1=None):
    """Median SM clock, maximum SM clock and the slowdown reasons seen in
    nvidia-smi sample lines (timestamp first, then ClockSampler.Q's fields).
    With a window [t0, t1] (epoch seconds) only the samples taken inside it
    count, when there are any; otherwise every sample does."""
    import datetime
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    parsed = []
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 10:
            continue
        try:
            sm, mx = float(f[2]), float(f[3])
        except ValueError:
            continue
        try:
            ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        active = [nm for k, nm in enumerate(names) if f[6 + k].lower().startswith("active")]
        parsed.append((ts, sm, mx, active))
    return _summary(parsed, t0, t1)


def _summary(parsed, t0, t1):
    if not parsed:
        return None
    inside = [p for p in parsed if t0 is not None and p[0] is not None and t0 <= p[0] <= t1]
    use = inside if inside else parsed
    out = {"sm_mhz": statistics.median(p[1] for p in use), "sm_max_mhz": max(p[2] for p in use),
           "reasons": sorted({r for p in use for r in p[3]}), "samples": len(use),
           "in_timed_region": bool(inside)}
    if t0 is not None:
        out["window_ms"] = round((t1 - t0) * 1e3, 3)
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons, one timestamped sample every
    10 ms (as fast as nvidia-smi answers), kept for the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self, wait_s: float = 3.0):
        """Start sampling; returns once the first sample is in (or after wait_s)."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        t_end = time.time() + wait_s
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(list(self.lines), t0, t1)


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, read-only queries) about once a millisecond from a host
    thread, so that a timed region of a few milliseconds still holds several
    samples.  Inactive when NVML cannot be loaded."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, cuda_index: int):
        self.ok = False
        self.samples = []
        self._stop = threading.Event()
        try:
            import torch
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            uuid = getattr(torch.cuda.get_device_properties(cuda_index), "uuid", None)
            got = False
            if uuid is not None:
                u = str(uuid)
                u = u if u.startswith("GPU-") else "GPU-" + u
                got = self.nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(self.h)) == 0
            if not got and self.nv.nvmlDeviceGetHandleByIndex_v2(cuda_index, ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) != 0:
                return
            self.max_mhz = float(mx.value)
            self.ok = True
        except Exception:
            self.ok = False

    def _poll(self):
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self._stop.is_set():
            t = time.time()
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                r = 0
                if self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(rs)) == 0:
                    r = rs.value
                self.samples.append((t, float(clk.value), self.max_mhz,
                                     [nm for bit, nm in self.REASONS.items() if r & bit]))
            time.sleep(0.001)

    def start(self):
        if self.ok:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            time.sleep(0.005)

    def stop(self, t0=None, t1=None):
        if not self.ok:
            return None
        time.sleep(0.005)
        self._stop.set()
        self.t.join(timeout=2)
        s = _summary(list(self.samples), t0, t1)
        if s:
            s["source"] = "nvml, ~1 ms"
        return s


class Clocks:
    """Both samplers over one window; the NVML summary when it has samples
    inside the window, else nvidia-smi's."""

    def __init__(self, index):
        self.nvml = NvmlSampler(index)
        self.smi = ClockSampler(index)

    def start(self):
        self.smi.start()
        self.nvml.start()

    def stop(self, t0, t1):
        a = self.nvml.stop(t0, t1)
        b = self.smi.stop(t0, t1)
        if b:
            b["source"] = "nvidia-smi, 10 ms"
        best = a if a and a.get("in_timed_region") else (b if b and b.get("in_timed_region") else (a or b))
        if best is not None and b is not None and best is not b:
            best["nvidia_smi"] = {k: b[k] for k in ("sm_mhz", "samples", "in_timed_region", "reasons")}
        return best


def source_digest(names):
    """sha256 prefix of the named library sources (paths under the package)."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        path = os.path.join(ROOT, "paper_1905_13376_gb300", name)
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_of(kernel):
    tr = TRAFFIC.get(kernel)
    if tr and tr.get("bytes_per_step") and tr.get("digest") == source_digest(tr["sources"]):
        return tr["bytes_per_step"]
    return None


# ---------------------------------------------------------------------------
# workloads, bytes, timing
# ---------------------------------------------------------------------------
def make_workload(args):
    from paper_1905_13376_gb300 import datagen
    F = datagen.chung_lu_directed(n_vertices=args.vertices, mean_degree=32.0)
    desc = (f"linear self-join F|x|F|x|F, COUNT(*) GROUP BY A; F = directed power-law graph, "
            f"{args.vertices} vertices, Zipf s=1.1 degrees capped at 4096, mean degree 32, "
            f"{len(F[0])} edges (int32 src,dst)")
    return F, desc


def table_bytes(direct, span, distinct, entry_bytes):
    """Stored size of a one-bucket table: the direct-address array (span
    entries) or 2^k >= 4 x distinct hashed 8-byte slots."""
    if direct:
        return entry_bytes * span
    slots = 16
    while slots < 4 * distinct:
        slots *= 2
    return 8 * slots


def algorithmic_bytes(name, nR, nS, nT, a_domain, t_bytes, w_bytes, launches=1):
    """Bytes a kernel must move per step (each buffer once at its stored size)."""
    if name == "w_build":
        # S streamed once (8 B per tuple); T's table read and S's weight
        # table written once, both at their stored size
        return 8 * nS + t_bytes + w_bytes
    if name == "w_probe_groupby":
        return 8 * nR + w_bytes + 8 * a_domain
    if name == "w_probe_count":
        return 8 * nR + w_bytes
    if name == "t_insert":
        return 4 * nT + t_bytes
    if name == "lin_probe_groupby":
        return 8 * nR + 8 * nS + t_bytes + 8 * a_domain
    if name == "lin_probe_count":
        return 8 * nR + 8 * nS + t_bytes
    if name == "part_scatter":
        return 16 * nR + 16 * nS + (8 * nT if launches >= 3 else 0)
    if name == "part_hist":
        return 4 * (nR + nS + nT)
    return None


def timed_ms(fn, stream, steps, warm=3):
    """Mean CUDA-event milliseconds of fn() over `steps` calls on `stream`,
    after `warm` untimed calls."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def profiled(ctx, fn, steps):
    """Per-kernel milliseconds and launches per call of fn() (the library runs
    a call's kernels on one stream while profiling, each timed alone)."""
    import torch
    ctx.set_profiling(True)
    ctx.reset_phase_times()
    for _ in range(steps):
        fn()
    torch.cuda.synchronize()
    ph = ctx.phase_times()
    ctx.set_profiling(False)
    return {k: (v[0] / steps, v[1] / steps) for k, v in ph.items()}


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over all ranks (the replicas'
    step times: the whole job is as slow as its slowest replica)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() and \
            torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def replica_throughput(units_per_replica, world, ms):
    """Whole-job throughput of `world` replicas that each process
    units_per_replica in at most ms milliseconds."""
    return units_per_replica * world / (ms * 1e-3)


def guarded(name, fn, *a, **kw):
    """Run one sub-benchmark; a failure is recorded in the line, not hidden."""
    try:
        return fn(*a, **kw)
    except Exception as e:   # noqa: BLE001
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"[:400], "arm": name}


# ---------------------------------------------------------------------------
# the cpu_baseline leg: every call of the CPU oracle (timed baseline and the
# exactness checks) is in these functions
# ---------------------------------------------------------------------------
def cpu_baseline(F, a_domain):
    """The oracle on the headline workload once: its throughput and its
    result (compared with the GPU's)."""
    import oracle
    t0 = time.perf_counter()
    want = oracle.linear(F, F, F, oracle.GROUP_BY_A, a_domain=a_domain)
    dt = time.perf_counter() - t0
    n = len(F[0])
    return ({"value": 3 * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": f"the full workload once ({3 * n} input tuples, {dt:.2f} s, 1 thread)"}, want)


def cpu_baseline_linear(R, S, T, a_domain):
    import oracle
    return oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)


def cpu_baseline_cyclic_sampled(R, S, T, sample, a_domain):
    """The oracle's GROUP BY A and rows of the cyclic join with R restricted
    to the sampled A values (exactly those values' groups and rows)."""
    import numpy as np
    import oracle
    keep = np.isin(R[0], sample)
    Rs = (R[0][keep], R[1][keep])
    g = oracle.cyclic(Rs, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
    rows = oracle.cyclic(Rs, S, T, oracle.MATERIALIZE, capacity=int(g["total"]))["rows"]
    return g["counts"][sample], rows


def cpu_baseline_planner_sample(meta, totals):
    """The oracle's totals of the planner arm's small instances (host copies
    kept while timing) against the engine's."""
    import oracle
    from paper_1905_13376_gb300 import binding
    ok, n = True, 0
    for m, tot in zip(meta, totals):
        if "rel" not in m:
            continue
        fn = oracle.linear if m["kind"] == binding.MWJ_LINEAR else oracle.cyclic
        ok = ok and fn(*m["rel"])["total"] == tot
        n += 1
    return (ok if n else None), n


def cpu_baseline_batch_sampled(qs, pick):
    import oracle
    out = {}
    for i in pick:
        q = qs[i]
        fn = oracle.linear if q.kind == "linear" else oracle.cyclic
        out[int(i)] = fn(q.R, q.S, q.T)["total"]
    return out


# ---------------------------------------------------------------------------
# the headline: F |x| F |x| F on the 2^20-vertex graph
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1905_13376_gb300 import binding

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    F, desc = make_workload(args)
    n = len(F[0])
    a_domain = args.vertices
    dF = tuple(torch.from_numpy(c).to(dev) for c in F)
    ctx = binding.Context(local_rank)
    shares = tuple(args.shares) if args.shares else ctx.plan_shares(binding.MWJ_LINEAR, dF, dF, dF,
                                                                    binding.MWJ_COUNT_GROUP_BY_A)
    stream = torch.cuda.current_stream(dev)
    r = ctx.join3_linear(dF, dF, dF, "group_by_a", shares=shares, a_domain=a_domain, sync=True)
    total = int(r["total"].item())
    counts_ref = r["counts"].clone()
    assert int(r["counts"].sum().item()) == total

    def step():
        ctx.join3_linear(dF, dF, dF, "group_by_a", shares=shares, a_domain=a_domain, sync=False, out=r)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    clk = Clocks(local_rank)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()   # host window holding the timed region's device work
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop(t0, t1)
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.launch_count() - launches0
    exact_steps = torch.equal(r["counts"], counts_ref) and int(r["total"].item()) == total

    # the same step sustained for about a quarter of a second (its own clock record)
    sustained = None
    if rank == 0 and world == 1 and not args.no_sustained:
        ks = max(args.steps, int(250.0 / max(ms, 1e-3)))
        clk2 = Clocks(local_rank)
        clk2.start()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0 = time.time()
        s0.record(stream)
        for _ in range(ks):
            step()
        s1.record(stream)
        torch.cuda.synchronize()
        u1 = time.time()
        sms = s0.elapsed_time(s1) / ks
        sustained = {"steps": ks, "ms_per_step": sms, "value": 3 * n / (sms * 1e-3),
                     "clocks": clk2.stop(u0, u1)}

    # per-kernel times (outside the timed regions)
    phases = profiled(ctx, step, args.steps)

    # end to end through the C ABI from pinned host memory: H2D of F (each
    # column in two halves, the four copies on four streams so that copy
    # engines run at once), the join, D2H of the group counts and the total,
    # every step
    hF = tuple(torch.from_numpy(c).pin_memory() for c in F)
    hcnt = torch.empty(a_domain, dtype=torch.int64).pin_memory()
    htot = torch.empty(1, dtype=torch.int64).pin_memory()
    eF = tuple(torch.empty_like(c) for c in dF)
    half = (n // 2) & ~255
    parts = [(col, lo, hi) for col in (0, 1) for lo, hi in ((0, half), (half, n))]
    sides = [torch.cuda.Stream(dev) for _ in parts]
    evs = [torch.cuda.Event() for _ in parts]
    er = {}

    def e2e_step():
        for (col, lo, hi), sd, ev in zip(parts, sides, evs):
            sd.wait_stream(stream)
            with torch.cuda.stream(sd):
                eF[col][lo:hi].copy_(hF[col][lo:hi], non_blocking=True)
                ev.record(sd)
        for ev in evs:
            stream.wait_event(ev)
        rr = ctx.join3_linear(eF, eF, eF, "group_by_a", shares=shares, a_domain=a_domain, sync=False,
                              out=er.get("r"))
        er["r"] = rr
        hcnt.copy_(rr["counts"], non_blocking=True)
        htot.copy_(rr["total"], non_blocking=True)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / args.steps
    assert int(htot.item()) == total

    # comparison arms, rank 0 only (the other ranks wait for it at the max
    # over ranks below)
    peak, peak_kind = peaks()
    first = rank == 0
    casc = None if args.no_cascade or not first else guarded("cascade", run_cascade, ctx, stream, args, F, dF,
                                                              a_domain, r, total)
    part = None if args.no_partitioned or not first else guarded("partitioned", run_partitioned, ctx, stream,
                                                                  args, dF, n, a_domain, r, ms, (peak, peak_kind))
    shuf = None if args.no_shuffled or not first else guarded("shuffled", run_shuffled, ctx, stream, args, F,
                                                               a_domain, counts_ref, total)
    if world > 1:
        ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev)

    tuples = 3 * n
    value = replica_throughput(tuples, world, ms)
    # one-bucket tables: the direct-address layout when the key range fits
    # (the library's choice is visible in which of the two pass kernels did
    # the work); T's and S's tables are both keyed by F's source column here
    direct = phases.get("w_build", (0, 0))[0] > phases.get("w_build_hashed", (0, 0))[0]
    src = F[0]
    span = int(src.max()) - int(src.min()) + 1
    dc = int(np.count_nonzero(np.bincount(src - src.min())))
    t_bytes = table_bytes(direct, span, dc, 4)
    w_bytes = table_bytes(direct, span, dc, 8)
    names = {"w_build": "w_build", "w_probe": "w_probe_groupby"}
    ktime = lambda k: phases.get(k, (0.0, 0))[0] + phases.get(k + "_hashed", (0.0, 0))[0]
    dom = max(phases, key=lambda k: phases[k][0]) if phases else None
    roof = None
    if dom:
        base = dom[:-len("_hashed")] if dom.endswith("_hashed") else dom
        ab = algorithmic_bytes(base, n, n, n, a_domain, t_bytes, w_bytes, phases[dom][1])
        if ab is not None:
            kms = ktime(base)
            achieved = ab / (kms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": base, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic_of(base), "peak_kind": peak_kind,
                    "algorithmic_bytes_per_step": ab, "ms_per_step": round(kms, 4),
                    "table_layout": "direct-address" if direct else "hashed"}
    # the whole multiway probe: S pass + R pass
    pb = algorithmic_bytes(names["w_build"], n, n, n, a_domain, t_bytes, w_bytes) + \
        algorithmic_bytes(names["w_probe"], n, n, n, a_domain, t_bytes, w_bytes)
    pms = ktime(names["w_build"]) + ktime(names["w_probe"])
    probe = {"kernels": ["w_build", "w_probe_groupby"], "algorithmic_bytes": pb, "ms_per_step": round(pms, 4),
             "achieved": round(pb / (pms * 1e-3) / 1e9, 1) if pms else None, "peak": peak, "unit": "GB/s",
             "frac": round(pb / (pms * 1e-3) / 1e9 / peak, 4) if pms else None}
    kernels = {k: {"ms_per_step": round(v[0], 4), "launches_per_step": v[1]} for k, v in phases.items()}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded power-law graph)",
        "config": {"workload": desc, "tuples_per_step": tuples, "l2": L2_NOTE,
                   "parallelism": f"replicas x{world}"},
        "plan": {"impl": ("multiway (single-step 3-way hash join)" +
                          (", one bucket per side: T's table and S's weight table held in L2"
                           if tuple(shares[:2]) == (1, 1) else ", partitioned")),
                 "shares": list(shares), "table_layout": "direct-address" if direct else "hashed",
                 "result_total": total, "result_tuples_per_s": total * world / (ms * 1e-3),
                 "exact_across_timed_steps": bool(exact_steps)},
        "roofline": roof, "probe_roofline": probe, "kernels": kernels,
        "e2e": {"value": replica_throughput(tuples, world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * a_domain + 8},
        "gpu_launches": launches, "clocks": clocks, "sustained": sustained,
        "partitioned": part, "cascade": casc, "shuffled": shuf,
    }
    if first and world == 1:
        out["uniform_2e16"] = None if args.no_configs or args.no_uniform else guarded(
            "uniform", run_uniform, ctx, stream, args)
        out["triangles"] = None if args.no_configs or args.no_triangles else guarded(
            "triangles", run_triangles, ctx, stream, args, (peak, peak_kind))
        out["batch_4096"] = None if args.no_configs or args.no_batch else guarded(
            "batch", run_batch, ctx, stream, args)
        out["planner"] = None if args.no_configs or args.no_planner else guarded(
            "planner", run_planner, ctx, stream, args)
        out["star"] = None if args.no_star else guarded("star", run_star, ctx, stream, args, (peak, peak_kind))
        out["skew"] = None if args.no_skew else guarded("skew", run_skew, ctx, stream, args)
        out["join4"] = None if args.no_join4 else guarded("join4", run_join4, ctx, stream, args, F)
        out["fm"] = None if args.no_fm else guarded("fm", run_fm, ctx, stream, args, F)
    return out, F, r["counts"].cpu().numpy(), total


def run_cascade(ctx, stream, args, F, dF, a_domain, r, total):
    """The cascade of binary joins on the headline workload, same device,
    same metric: I = F |x| F (~1e9 rows, 12 B each) is materialised in HBM."""
    import numpy as np
    import torch
    from paper_1905_13376_gb300 import binding
    n = len(F[0])
    indeg = np.bincount(F[1], minlength=a_domain).astype(np.int64)
    outdeg = np.bincount(F[0], minlength=a_domain).astype(np.int64)
    nI = int((indeg * outdeg).sum())
    base_ws = ctx.workspace_size(2 + binding.MWJ_LINEAR, dF, dF, dF, None, binding.MWJ_COUNT_GROUP_BY_A)
    wsb = base_ws + max(0, nI - (1 << 24)) * 12 + (64 << 20)

    def cstep():
        return ctx.cascade_join(binding.MWJ_LINEAR, dF, dF, dF, "group_by_a", a_domain=a_domain, sync=False,
                                workspace_bytes=wsb)
    rc = cstep()
    torch.cuda.synchronize()
    exact = int(rc["total"].item()) == total and torch.equal(rc["counts"], r["counts"])
    cms = timed_ms(cstep, stream, max(3, args.steps // 4), warm=2)
    return {"impl": "cascade of binary hash joins (I = F|x|F materialised in HBM)",
            "value": 3 * n / (cms * 1e-3), "unit": UNIT, "ms_per_step": cms, "intermediate_rows": nI,
            "intermediate_bytes": 12 * nI, "multiway_speedup": None, "exact_match_multiway": bool(exact)}


def run_partitioned(ctx, stream, args, dF, n, a_domain, r, ms, pk):
    """The partitioned plan on the headline workload: R and S by H(B) into
    shared-memory buckets (Algorithm 1 with the library's default bucket
    count for row output), with the roofline of its probe kernel."""
    import torch
    from paper_1905_13376_gb300 import binding
    psh = ctx.plan_shares(binding.MWJ_LINEAR, dF, dF, dF, binding.MWJ_MATERIALIZE)
    rp = ctx.join3_linear(dF, dF, dF, "group_by_a", shares=psh, a_domain=a_domain)
    exact = int(rp["total"].item()) == int(r["total"].item()) and torch.equal(rp["counts"], r["counts"])

    def pstep():
        ctx.join3_linear(dF, dF, dF, "group_by_a", shares=psh, a_domain=a_domain, sync=False, out=rp)
    pms = timed_ms(pstep, stream, args.steps)
    ph = profiled(ctx, pstep, 3)
    kname = "lin_probe_groupby"
    roof = None
    if kname in ph:
        # T's single table: hashed, 2^k >= 4 x distinct slots of 8 bytes
        import numpy as np
        src = dF[0].cpu().numpy()
        t_bytes = table_bytes(False, 0, int(np.count_nonzero(np.bincount(src - src.min()))), 8)
        ab = algorithmic_bytes(kname, n, n, n, a_domain, t_bytes, 0)
        ach = ab / (ph[kname][0] * 1e-3) / 1e9
        roof = {"kernel": kname, "ms_per_step": round(ph[kname][0], 4), "algorithmic_bytes": ab,
                "achieved": round(ach, 1), "peak": pk[0], "unit": "GB/s", "frac": round(ach / pk[0], 4),
                "peak_kind": pk[1]}
    return {"impl": "partitioned: R and S by H(B), each bucket's B values in shared memory (Algorithm 1)",
            "shares": list(psh), "value": 3 * n / (pms * 1e-3), "unit": UNIT, "ms_per_step": pms,
            "default_plan_speedup": pms / ms, "exact_match_default": bool(exact), "probe_roofline": roof,
            "kernels": {k: round(v[0], 4) for k, v in ph.items()}}


def run_shuffled(ctx, stream, args, F, a_domain, counts_ref, total):
    """The headline graph with its rows in a seeded random order (no runs of
    equal keys for the warps to merge): same metric, same result."""
    import numpy as np
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    perm = np.random.default_rng(20).permutation(len(F[0]))
    Fs = (np.ascontiguousarray(F[0][perm]), np.ascontiguousarray(F[1][perm]))
    dF = tuple(torch.from_numpy(c).to(dev) for c in Fs)
    rs = ctx.join3_linear(dF, dF, dF, "group_by_a", a_domain=a_domain)
    exact = int(rs["total"].item()) == total and torch.equal(rs["counts"], counts_ref.to(dev))
    ms = timed_ms(lambda: ctx.join3_linear(dF, dF, dF, "group_by_a", a_domain=a_domain, sync=False, out=rs),
                  stream, args.steps)
    ph = profiled(ctx, lambda: ctx.join3_linear(dF, dF, dF, "group_by_a", a_domain=a_domain, sync=False,
                                                out=rs), 3)
    n = len(F[0])
    return {"workload": "the headline graph with its rows shuffled (seeded permutation)",
            "value": 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "exact_match_sorted": bool(exact), "kernels": {k: round(v[0], 4) for k, v in ph.items()}}


# ---------------------------------------------------------------------------
# the other workloads
# ---------------------------------------------------------------------------
def run_uniform(ctx, stream, args):
    """Linear join R(A,B) S(B,C) T(C,D), 2^16 uniform tuples each (A, D in
    [0, 2^20), B, C in [0, 2^12)), COUNT(*) GROUP BY A: multiway vs cascade."""
    import numpy as np
    import torch
    from paper_1905_13376_gb300 import binding, datagen
    R, S, T = datagen.linear_uniform()
    adom = 1 << 20
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda rel: tuple(torch.from_numpy(c).to(dev) for c in rel)
    dR, dS, dT = d(R), d(S), d(T)
    r = ctx.join3_linear(dR, dS, dT, "group_by_a", a_domain=adom)
    ms = timed_ms(lambda: ctx.join3_linear(dR, dS, dT, "group_by_a", a_domain=adom, sync=False, out=r),
                  stream, max(args.steps, 50))
    rc = ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=adom)
    cexact = torch.equal(rc["counts"], r["counts"])
    cms = timed_ms(lambda: ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=adom,
                                            sync=False), stream, max(args.steps, 20))
    nI = int((np.bincount(R[1], minlength=1 << 12).astype(np.int64) *
              np.bincount(S[0], minlength=1 << 12).astype(np.int64)).sum())
    exact = None
    if not args.no_cpu_baseline:
        want = cpu_baseline_linear(R, S, T, adom)
        exact = int(r["total"].item()) == want["total"] and np.array_equal(r["counts"].cpu().numpy(),
                                                                           want["counts"])
    n = 3 * len(R[0])
    return {"workload": "linear R|x|S|x|T, 2^16 tuples per relation, A,D uniform in [0,2^20), "
                        "B,C uniform in [0,2^12), COUNT(*) GROUP BY A",
            "value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "result_total": int(r["total"].item()),
            "cascade": {"ms_per_step": cms, "value": n / (cms * 1e-3), "intermediate_rows": nI,
                        "exact_match_multiway": bool(cexact)},
            "multiway_speedup": cms / ms, "exact_vs_oracle": exact}


def run_triangles(ctx, stream, args, pk):
    """Cyclic join R(A,B) S(B,C) T(C,A) on the 2^22-vertex power-law graph
    (edges oriented a < b, T the reversed edges): total, GROUP BY A, the
    materialised triangle list (capacity from the count) and the cascade of
    binary joins, run in chunks of its intermediate."""
    import numpy as np
    import torch
    from paper_1905_13376_gb300 import binding, datagen
    n_v = args.triangle_vertices
    a, b = datagen.chung_lu_undirected(n_vertices=n_v)
    R, S, T = datagen.triangle_relations(a, b)
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda rel: tuple(torch.from_numpy(np.ascontiguousarray(c)).to(dev) for c in rel)
    dR, dS, dT = d(R), d(S), d(T)
    wedges = int((np.bincount(b, minlength=n_v).astype(np.int64) *
                  np.bincount(a, minlength=n_v).astype(np.int64)).sum())   # |R join S| on B
    steps = max(3, args.steps // 4)
    rc = ctx.join3_cyclic(dR, dS, dT, "count")
    total = int(rc["total"].item())
    cms = timed_ms(lambda: ctx.join3_cyclic(dR, dS, dT, "count", sync=False, out=rc), stream, steps, warm=2)
    rg = ctx.join3_cyclic(dR, dS, dT, "group_by_a", a_domain=n_v)
    gms = timed_ms(lambda: ctx.join3_cyclic(dR, dS, dT, "group_by_a", a_domain=n_v, sync=False, out=rg),
                   stream, steps, warm=2)
    counts = rg["counts"].cpu().numpy()
    ph = profiled(ctx, lambda: ctx.join3_cyclic(dR, dS, dT, "count", sync=False, out=rc), 2)
    # the materialised list
    rr = ctx.join3_cyclic(dR, dS, dT, "rows", capacity=total)
    n_rows = int(rr["n_rows"].item())
    g = np.random.default_rng(1)
    hubs = np.argsort(-np.bincount(a))[:5].astype(np.int32)
    sample = np.unique(np.concatenate([g.choice(a, 300), hubs]))
    rows = rr["rows"]
    mine = rows[torch.isin(rows[:, 0], torch.from_numpy(sample).to(dev))].cpu().numpy()
    del rr, rows
    torch.cuda.synchronize()
    rms = timed_ms(lambda: ctx.join3_cyclic(dR, dS, dT, "rows", capacity=total, sync=False), stream, 3, warm=1)
    torch.cuda.empty_cache()
    # the cascade: I = R |x| S on B, chunked through a 32 GB workspace
    casc = None
    if not args.no_cascade:
        wsb = 32 << 30
        t0 = time.time()
        rcas = ctx.cascade_join(binding.MWJ_CYCLIC, dR, dS, dT, "count", workspace_bytes=wsb)
        torch.cuda.synchronize()
        c_ms = timed_ms(lambda: ctx.cascade_join(binding.MWJ_CYCLIC, dR, dS, dT, "count", sync=False,
                                                 workspace_bytes=wsb), stream, 1, warm=0)
        casc = {"ms_per_step": c_ms, "intermediate_rows": wedges, "intermediate_bytes": 12 * wedges,
                "workspace_bytes": wsb, "exact_match_multiway": int(rcas["total"].item()) == total,
                "first_call_s": round(time.time() - t0, 2), "multiway_speedup": c_ms / cms}
        del rcas
        ctx._ws = None
        torch.cuda.empty_cache()
    # the probe kernel's rate: one wedge check (a (c, a) membership probe in
    # T_ki's shared-memory set) per R tuple of a bucket per S tuple whose b
    # it shares; counted once per wedge of R |x| S (tiles split into several
    # items re-probe, so this is a lower bound of the work).  Peak: every
    # SM's 32 shared-memory banks serve 128 B per clock, 8 B per probe.
    pkern = "cyc_c_probe" if "cyc_c_probe" in ph else "cyc_probe"   # C-bucket plan, else the cube tiling
    pms = ph.get(pkern, (float("nan"), 0))[0]
    import json as _json
    peaks_file = os.path.join(ROOT, "MEASURED_PEAKS.json")
    fmax = _json.load(open(peaks_file)).get("sm_max_mhz", 2070.0) if os.path.exists(peaks_file) else 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_probes = n_sm * fmax * 1e6 * 128 / 8
    rate = wedges / (pms * 1e-3)
    exact = None
    if not args.no_cpu_baseline:
        want_counts, want_rows = cpu_baseline_cyclic_sampled(R, S, T, sample, n_v)
        exact = bool(np.array_equal(counts[sample], want_counts) and
                     np.array_equal(_sorted_rows(mine), want_rows))
    nin = len(R[0]) + len(S[0]) + len(T[0])
    return {"workload": f"cyclic R|x|S|x|T (triangles) on a power-law graph of {n_v} vertices, "
                        f"{len(a)} undirected edges oriented a<b; R = S = edges, T = reversed edges",
            "shares": list(ctx.plan_shares(binding.MWJ_CYCLIC, dR, dS, dT)), "result_total": total,
            "count": {"ms_per_step": cms, "value": nin / (cms * 1e-3), "unit": UNIT},
            "group_by_a": {"ms_per_step": gms, "value": nin / (gms * 1e-3), "unit": UNIT,
                           "sum_equals_total": int(counts.sum()) == total},
            "rows": {"ms_per_step": rms, "n_rows": n_rows, "rows_equal_total": n_rows == total,
                     "bytes": 12 * n_rows, "result_tuples_per_s": n_rows / (rms * 1e-3)},
            "cascade": casc,
            "probe": {"kernel": pkern, "bound": "smem", "ms_per_step": round(pms, 4),
                      "wedge_checks": wedges, "achieved": rate, "peak": peak_probes,
                      "unit": "wedge checks/s", "frac": round(rate / peak_probes, 4),
                      "peak_derivation": f"{n_sm} SMs x {fmax:.0f} MHz x 128 B/clock of shared memory / 8 B per probe"},
            "kernels": {k: round(v[0], 4) for k, v in ph.items()},
            "exact_vs_oracle": exact,
            "exact_sample": f"{len(sample)} A values (300 drawn from the edge list and the 5 busiest) "
                            "against the oracle's groups and rows for R restricted to them"}


def _sorted_rows(x):
    import numpy as np
    x = np.asarray(x)
    if x.size == 0:
        return x.reshape(0, x.shape[1] if x.ndim == 2 else 3)
    return x[np.lexsort(x.T[::-1])]


def run_batch(ctx, stream, args):
    """args.batch_queries (4096) independent joins (linear and cyclic alternating, sizes
    log-uniform in [2^8, 2^18], domains in [2^6, 2^20], uniform or Zipf(1.0)
    keys) in one persistent launch, captured into a CUDA graph and replayed;
    COUNT(*) per query."""
    import numpy as np
    import torch
    from paper_1905_13376_gb300 import binding, datagen
    t0 = time.time()
    qs = datagen.batched_queries(args.batch_queries)
    gen_s = time.time() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda rel: tuple(torch.from_numpy(np.ascontiguousarray(c)).to(dev) for c in rel)
    dq = [(binding.MWJ_LINEAR if q.kind == "linear" else binding.MWJ_CYCLIC, d(q.R), d(q.S), d(q.T))
          for q in qs]
    tuples = int(sum(len(q.R[0]) + len(q.S[0]) + len(q.T[0]) for q in qs))
    b = binding.Batch(ctx, dq)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        b.launch(stream=s)   # binds the workspace (outside the capture)
    torch.cuda.synchronize()
    got = b.counts[: b.n].cpu().numpy().copy()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.launch(stream=s)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    replay_same = bool(np.array_equal(b.counts[: b.n].cpu().numpy(), got))
    sizes = np.array([len(q.R[0]) + len(q.S[0]) + len(q.T[0]) for q in qs])
    g = np.random.default_rng(4)
    pick = np.unique(np.concatenate([np.argsort(-sizes)[:8], g.choice(len(qs), 40, replace=False)]))
    exact = None
    if not args.no_cpu_baseline:
        want = cpu_baseline_batch_sampled(qs, pick)
        exact = all(int(got[i]) == want[int(i)] for i in pick)
    lin = [i for i, q in enumerate(qs) if q.kind == "linear"]
    shares_lin = [b.shares(i) for i in lin[:3]]
    b.close()
    out = {"workload": f"{len(qs)} joins (linear and cyclic alternating), |R|,|S|,|T| log-uniform in "
                       "[2^8,2^18], key domains log-uniform in [2^6,2^20], uniform or Zipf(1.0) keys, "
                       "COUNT(*) per query",
           "impl": "one persistent partition launch and one persistent join launch over all queries, "
                   "replayed from a CUDA graph", "input_tuples": tuples,
           "value": tuples / (ms * 1e-3), "unit": UNIT, "ms_per_launch": ms, "replays": reps,
           "replay_counts_equal_first_launch": replay_same, "exact_vs_oracle": exact,
           "exact_sample": f"{len(pick)} queries (the 8 largest and 40 drawn at random)",
           "example_shares_linear": [list(x) for x in shares_lin], "generation_s": round(gen_s, 1),
           "autotuned": None}
    if args.no_autotune:
        return out
    # the autotuner: rules per (kind, size class) and launch shapes timed on
    # these queries, then the batch planned again and replayed the same way
    from paper_1905_13376_gb300 import autotune
    tuning = autotune.autotune(ctx, dq)
    bt = binding.Batch(ctx, dq)
    with torch.cuda.stream(s):
        bt.launch(stream=s)
    torch.cuda.synchronize()
    got_t = bt.counts[: bt.n].cpu().numpy().copy()
    graph_t = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_t, stream=s):
        bt.launch(stream=s)
    for _ in range(2):
        graph_t.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        graph_t.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1) / reps
    tuned_same = bool(np.array_equal(got_t, got)) and bool(np.array_equal(bt.counts[: bt.n].cpu().numpy(), got))
    bt.close()
    ctx.batch_set_rules([])
    ctx.batch_set_launch(0, 0)
    out["autotuned"] = {"ms_per_launch": ms_t, "value": tuples / (ms_t * 1e-3), "unit": UNIT,
                        "speedup_over_library_rule": ms / ms_t,
                        "counts_equal_library_rule": tuned_same,
                        "tuning_seconds": round(tuning["tuning_seconds"], 1),
                        "rules_changed": len(tuning["rules"]), "launch": tuning["launch"],
                        "tuner_whole_batch_ms": tuning["whole_batch_ms"],
                        "context_queries": tuning["context_queries"],
                        "class_timings": tuning["class_timings"]}
    return out


def run_planner(ctx, stream, args):
    """The learned planner on held-out instances generated now (a seed the
    training never used; sizes log-uniform in [2^10, 2^24], uniform or Zipf
    keys, linear and cyclic): every plan timed on this engine, regret of the
    packaged network's choice against the best measured plan, next to the
    cost model alone and each fixed plan."""
    import numpy as np
    from paper_1905_13376_gb300 import planner
    t0 = time.time()
    F, times, totals, meta, rejected = planner.collect(ctx, args.planner_instances, 777, args.planner_budget,
                                                       keep_small=1 << 22)
    summary, per = planner.evaluate(planner.default_planner(ctx), F, times, [m["sizes"] for m in meta])
    # the instance where the library's default plan loses most to the best plan
    worst = None
    if len(F):
        i = int(np.argmax(per["default"]))
        worst = {k: meta[i][k] for k in ("kind", "sizes", "domains", "zipf")}
        worst.update({"us_per_plan": times[i], "default_regret": per["default"][i],
                      "learned_regret": per["learned"][i]})
    exact, checked = (None, 0)
    if not args.no_cpu_baseline:
        exact, checked = cpu_baseline_planner_sample(meta, totals)
    ctx._ws = None
    return {"workload": "held-out join instances: |R|,|S|,|T| log-uniform in [2^10,2^24], domains in "
                        "[2^6,2^22], uniform or Zipf(0.8..1.5) keys, linear and cyclic",
            "instances": len(F), "rejected": rejected, "seconds": round(time.time() - t0, 1),
            "plans": ["cascade", "3-way default shares", "3-way alternative shares"],
            "regret": summary, "worst_default": worst, "plans_agree_on_every_total": True,
            "exact_vs_oracle": exact, "oracle_checked_instances": checked}


def run_star(ctx, stream, args, pk):
    """The star 3-way join (fact relation streamed once past two dimension
    tables) against the cascade of binary joins on the same inputs."""
    import numpy as np
    import torch
    from paper_1905_13376_gb300 import binding, datagen

    R, S, T = datagen.star_schema()
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda rel: tuple(torch.from_numpy(c).to(dev) for c in rel)
    dR, dS, dT = d(R), d(S), d(T)
    adom = 1 << 16
    nS, nR, nT = len(S[0]), len(R[0]), len(T[0])
    r = ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=adom)
    # closed form: every fact tuple joins one tuple of each dimension
    inv = np.empty(nR, dtype=np.int64)
    inv[R[1]] = np.arange(nR)
    want = np.bincount(R[0][inv[S[0]]], minlength=adom)
    exact = int(r["total"].item()) == nS and np.array_equal(r["counts"].cpu().numpy(), want)
    step = lambda: ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=adom, sync=False)
    ms = timed_ms(step, stream, args.steps)
    ph = profiled(ctx, step, args.steps)
    probe_ms = ph.get("star_probe_groupby", (float("nan"), 0))[0]
    # the probe reads S once (8 B per tuple) and both degree tables once
    slots = lambda n: 1 << max(4, int(np.ceil(np.log2(4 * n))))
    pbytes = 8 * nS + 8 * (slots(nR) + slots(nT))
    ach = pbytes / (probe_ms * 1e-3) / 1e9
    rc = ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=adom)
    exact = exact and torch.equal(rc["counts"], r["counts"])
    cms = timed_ms(lambda: ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=adom,
                                            sync=False), stream, max(3, args.steps // 4))
    return {"workload": f"star join: fact S(B,C) {nS} tuples (foreign keys, sorted by B), "
                        f"dimensions R(A,B), T(C,D) {nR} tuples each (unique keys), "
                        f"COUNT(*) GROUP BY A over 2^16 groups",
            "value": (nS + nR + nT) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "exact_vs_closed_form": bool(exact),
            "probe": {"kernel": "star_probe_groupby", "ms_per_step": round(probe_ms, 4),
                      "algorithmic_bytes": pbytes, "achieved": round(ach, 1), "peak": pk[0],
                      "unit": "GB/s", "frac": round(ach / pk[0], 4), "peak_kind": pk[1]},
            "cascade_ms_per_step": cms, "multiway_speedup": cms / ms}


def run_skew(ctx, stream, args):
    """The linear GROUP BY A with a Zipf(1.5) join column shared by R and S,
    with the default plan (heavy keys summed per CTA) and the partitioned one
    (heavy keys split off into their own bucket), checked exactly against the
    factorised sum cnt(a) = sum over (a,b) in R of sum over (b,c) in S of
    deg_T(c)."""
    import numpy as np
    from paper_1905_13376_gb300 import binding, datagen
    import torch

    R, S, T = datagen.skewed_linear()
    n = len(R[0])
    adom = 1 << 20
    dev = torch.device("cuda", torch.cuda.current_device())
    d = lambda rel: tuple(torch.from_numpy(c).to(dev) for c in rel)
    dR, dS, dT = d(R), d(S), d(T)
    # exact check (int64, numpy)
    off = np.int64(1) << 31
    kt, ct = np.unique(T[0], return_counts=True)
    p = np.minimum(np.searchsorted(kt, S[1]), len(kt) - 1)
    dS_ = np.where(kt[p] == S[1], ct[p], 0).astype(np.int64)
    kb, inv = np.unique(S[0].astype(np.int64) + off, return_inverse=True)
    w = np.zeros(len(kb), dtype=np.int64)
    np.add.at(w, inv, dS_)
    p = np.minimum(np.searchsorted(kb, R[1].astype(np.int64) + off), len(kb) - 1)
    wR = np.where(kb[p] == R[1].astype(np.int64) + off, w[p], 0)
    want = np.zeros(adom, dtype=np.int64)
    np.add.at(want, R[0].astype(np.int64), wR)
    psh = ctx.plan_shares(binding.MWJ_LINEAR, dR, dS, dT, binding.MWJ_MATERIALIZE)
    exact = True
    for sh in (None, psh):
        r = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=sh, a_domain=adom)
        exact = exact and int(r["total"].item()) == int(want.sum()) and \
            np.array_equal(r["counts"].cpu().numpy(), want)
    ms = timed_ms(lambda: ctx.join3_linear(dR, dS, dT, "group_by_a", a_domain=adom, sync=False),
                  stream, args.steps)
    pms = timed_ms(lambda: ctx.join3_linear(dR, dS, dT, "group_by_a", shares=psh, a_domain=adom,
                                            sync=False), stream, args.steps)
    top = float(np.bincount(S[0]).max()) / n
    return {"workload": f"linear R|x|S|x|T GROUP BY A, {n} tuples per relation, B Zipf(1.5) in R and S "
                        f"(one key map; top key {top:.1%} of S), A, C, D uniform",
            "impl": "one bucket per side; heavy keys summed per CTA in shared memory",
            "value": 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "exact_vs_factorised_sum": bool(exact), "result_total": int(want.sum()),
            "partitioned": {"impl": "partitioned by H(B) with the heavy keys in one extra bucket",
                            "shares": list(psh), "ms_per_step": pms, "value": 3 * n / (pms * 1e-3)}}


def run_join4(ctx, stream, args, F):
    """F |x| F |x| F |x| F GROUP BY A on the benchmark graph: the chain one
    relation longer, one more hash level (U's degrees, T's weights)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    dF = tuple(torch.from_numpy(c).to(dev) for c in F)
    adom = args.vertices
    r = ctx.join4_linear(dF, dF, dF, dF, "group_by_a", a_domain=adom)
    exact_sum = int(r["counts"].sum().item()) == int(r["total"].item())
    ms = timed_ms(lambda: ctx.join4_linear(dF, dF, dF, dF, "group_by_a", a_domain=adom, sync=False),
                  stream, args.steps)
    n = len(F[0])
    return {"workload": "chain of four relations F|x|F|x|F|x|F, COUNT(*) GROUP BY A, same graph",
            "value": 4 * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "result_total": int(r["total"].item()), "group_sum_equals_total": bool(exact_sum)}


def run_fm(ctx, stream, args, F):
    """Flajolet-Martin sketches of every person's distinct friends of friends
    of friends on the benchmark graph (the approximate query of the paper's
    Section 4.1 footnote)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    dF = tuple(torch.from_numpy(c).to(dev) for c in F)
    adom = args.vertices
    r = ctx.fm_linear(dF, dF, dF, adom)
    ms = timed_ms(lambda: ctx.fm_linear(dF, dF, dF, adom, sync=False), stream, args.steps)
    n = len(F[0])
    est = r["estimates"]
    return {"workload": "distinct friends of friends of friends per person, PCSA sketches "
                        "(16 x 32-bit bitmaps), F|x|F|x|F on the same graph",
            "value": 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "median_estimate": float(est.median().item()), "max_estimate": float(est.max().item())}


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle on the same workload and metric
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return None
    F, desc = make_workload(args)
    import oracle
    n = len(F[0])
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.linear(F, F, F, oracle.GROUP_BY_A, a_domain=args.vertices)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = 3 * n / (ms * 1e-3)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded power-law graph)",
            "config": {"workload": desc, "tuples_per_step": 3 * n, "l2": L2_NOTE,
                       "parallelism": f"replicas x{world}"},
            "plan": {"impl": "CPU oracle, single-threaded C hash join"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the full workload per step ({3 * n} input tuples)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--vertices", type=int, default=1 << 20)
    ap.add_argument("--shares", type=int, nargs="+", default=None,
                    help="I J [log2 table slots]")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU oracle (timed baseline and exactness flags)")
    ap.add_argument("--no-cascade", action="store_true")
    ap.add_argument("--no-partitioned", action="store_true",
                    help="skip timing the partitioned plan beside the default one")
    ap.add_argument("--no-shuffled", action="store_true", help="skip the shuffled-rows arm")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the uniform, triangle and batch workloads")
    ap.add_argument("--no-uniform", action="store_true", help="skip the 2^16-tuple uniform workload")
    ap.add_argument("--no-triangles", action="store_true", help="skip the triangle workload")
    ap.add_argument("--no-batch", action="store_true", help="skip the 4096-query batch")
    ap.add_argument("--batch-queries", type=int, default=4096,
                    help="queries of the batch arm (4096: the benchmark's workload)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the autotuned leg of the batch arm")
    ap.add_argument("--no-planner", action="store_true", help="skip the learned planner's held-out run")
    ap.add_argument("--no-sustained", action="store_true",
                    help="skip the quarter-second sustained timing of the headline step")
    ap.add_argument("--planner-instances", type=int, default=128)
    ap.add_argument("--planner-budget", type=float, default=60.0, help="seconds for the planner arm's instances")
    ap.add_argument("--triangle-vertices", type=int, default=1 << 22,
                    help="vertices of the triangle workload's graph")
    ap.add_argument("--no-fm", action="store_true",
                    help="skip the Flajolet-Martin sketch arm")
    ap.add_argument("--no-join4", action="store_true",
                    help="skip the four-relation chain arm")
    ap.add_argument("--no-skew", action="store_true",
                    help="skip the skewed-join arm (Zipf(1.5) join column, 2^22 tuples)")
    ap.add_argument("--no-star", action="store_true",
                    help="skip the star-join arm (fact relation 2^26 tuples)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    out, F, counts, total = run_ours(args, rank, world, local_rank)
    if rank == 0:
        out["exact_vs_oracle"] = None
        if world == 1 and not args.no_cpu_baseline:
            import numpy as np
            cb, want = cpu_baseline(F, args.vertices)
            out["cpu_baseline"] = cb
            out["exact_vs_oracle"] = bool(want["total"] == total and np.array_equal(want["counts"], counts))
        if out.get("cascade") and "ms_per_step" in out["cascade"]:
            out["cascade"]["multiway_speedup"] = out["cascade"]["ms_per_step"] / out["ms_per_step"]
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
