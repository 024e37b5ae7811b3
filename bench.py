#!/usr/bin/env python
"""Benchmark of the GB300 3-way hash join: input tuples/s of the linear
friends-of-friends-of-friends self-join F |x| F |x| F (COUNT(*) GROUP BY A)
on a synthetic power-law graph of 2^20 vertices (Zipf s=1.1 degrees capped at
4096, mean degree 32, ~3.3e7 directed edges), multiway vs cascade, exact
counts.

Prints one JSON line.  `python bench.py --gpus N --steps K --warmup W`; under
torchrun every rank runs its own replica of the workload (the join is one
problem per GPU; replicas only) and rank 0 reports the aggregate.

--impl reference times the CPU oracle (single-threaded C hash join) on the
same workload and metric.
"""
from __future__ import annotations

import argparse
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

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel from
# one ncu capture, per step of the benchmark workload, valid while the sources
# the kernel is built from are unchanged (digest of those files).  The
# scatter's capture ran on the 2^19-vertex graph (16,090,397 edges: S's and R's
# scatter moved 215.5 + 260.6 MB) and is scaled by the edge count to the
# 2^20-vertex graph (32,804,288 edges, x 2.0387): traffic grows with the tuples
# partitioned (the bucket count is the same).
# The one-bucket S pass (w_build) was captured the same way on the 2^19-vertex
# graph (162.3 MB read + 5.0 MB written) and scaled by the same factor (its
# tables double with the vertex count as well).
TRAFFIC = {
    "part_scatter": {"bytes_per_step": 970_700_000, "digest": "a8955b800db65c70",
                     "sources": ["csrc/partition.cu", "csrc/common.cuh", "csrc/internal.h", "csrc/skew.h"]},
    "w_build": {"bytes_per_step": 341_100_000, "digest": "6a71c3e30d2a52f4",
                "sources": ["csrc/linear_l2.cu", "csrc/linear_l2.h", "csrc/common.cuh", "csrc/internal.h",
                            "csrc/skew.h", "csrc/tables.h"]},
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


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


def make_workload(args):
    from paper_1905_13376_gb300 import datagen
    F = datagen.chung_lu_directed(n_vertices=args.vertices, mean_degree=32.0)
    desc = (f"linear self-join F|x|F|x|F, COUNT(*) GROUP BY A; F = directed power-law graph, "
            f"{args.vertices} vertices, Zipf s=1.1 degrees capped at 4096, mean degree 32, "
            f"{len(F[0])} edges (int32 src,dst)")
    return F, desc


def algorithmic_bytes(name, nR, nS, nT, a_domain, tslots, launches, wslots=0):
    """Bytes a kernel must move per step (each buffer once at its stored size)."""
    if name == "w_build":
        # S streamed once (8 B per tuple); T's table read and S's weight
        # table written once, both at their stored size
        return 8 * nS + 8 * tslots + 8 * wslots
    if name == "w_probe_groupby":
        return 8 * nR + 8 * wslots + 8 * a_domain
    if name == "w_probe_count":
        return 8 * nR + 8 * wslots
    if name == "t_insert":
        return 4 * nT + 8 * tslots
    if name == "lin_probe_groupby":
        return 8 * nR + 8 * nS + 8 * tslots + 8 * a_domain
    if name == "lin_probe_count":
        return 8 * nR + 8 * nS + 8 * tslots
    if name == "part_scatter":
        # R and S: read 8 B + write 8 B per tuple; T (keys only, when it is
        # partitioned: a third launch) read 4 + write 4
        return 16 * nR + 16 * nS + (8 * nT if launches >= 3 else 0)
    if name == "part_hist":
        return 4 * (nR + nS + nT)
    if name == "t_aggregate":
        return 4 * nT + 8 * nT
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

    def step(sync=False):
        return ctx.join3_linear(dF, dF, dF, "group_by_a", shares=shares, a_domain=a_domain,
                                sync=sync)

    # exactness check once (device result vs the oracle is in the tests; here
    # the group counts must at least sum to the total)
    r = step(sync=True)
    total = int(r["total"].item())
    assert int(r["counts"].sum().item()) == total
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    clk = ClockSampler(local_rank)
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
    # per-kernel times: the same steps again with an event pair around every
    # launch (outside the timed region above; the library runs them on one
    # stream while profiling, so each kernel is timed alone)
    ctx.set_profiling(True)
    ctx.reset_phase_times()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    phases = ctx.phase_times()
    ctx.set_profiling(False)

    # end to end through the C ABI from pinned host memory: H2D of F, the
    # join, D2H of the group counts and the total, every step
    hF = tuple(torch.from_numpy(c).pin_memory() for c in F)
    hcnt = torch.empty(a_domain, dtype=torch.int64).pin_memory()
    htot = torch.empty(1, dtype=torch.int64).pin_memory()
    eF = tuple(torch.empty_like(c) for c in dF)

    def e2e_step():
        for h, d in zip(hF, eF):
            d.copy_(h, non_blocking=True)
        rr = ctx.join3_linear(eF, eF, eF, "group_by_a", shares=shares, a_domain=a_domain,
                              sync=False)
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

    # the cascade of binary joins on the same workload, same device, same
    # metric: I = F|x|F (~1e9 rows, 12 B each) is materialised in HBM
    # the comparison arms run once, on rank 0 (the other ranks wait for it at
    # the max over ranks below)
    casc = None
    if not args.no_cascade and rank == 0:
        # room for I: the exact |F|x|F| from degrees (host, numpy)
        indeg = np.bincount(F[1], minlength=a_domain).astype(np.int64)
        outdeg = np.bincount(F[0], minlength=a_domain).astype(np.int64)
        nI = int((indeg * outdeg).sum())
        base_ws = ctx.workspace_size(2 + binding.MWJ_LINEAR, dF, dF, dF, None,
                                     binding.MWJ_COUNT_GROUP_BY_A)
        wsb = base_ws + max(0, nI - (1 << 24)) * 12 + (64 << 20)

        def cstep():
            return ctx.cascade_join(binding.MWJ_LINEAR, dF, dF, dF, "group_by_a",
                                    a_domain=a_domain, sync=False, workspace_bytes=wsb)
        rc = cstep()
        torch.cuda.synchronize()
        assert int(rc["total"].item()) == total
        assert torch.equal(rc["counts"], r["counts"])
        for _ in range(2):
            cstep()
        torch.cuda.synchronize()
        csteps = max(3, args.steps // 4)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(csteps):
            cstep()
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / csteps
        casc = {"impl": "cascade of binary hash joins (I = F|x|F materialised in HBM)",
                "value": 3 * n / (cms * 1e-3), "unit": UNIT, "ms_per_step": cms,
                "intermediate_rows": nI, "intermediate_bytes": 12 * nI, "steps": csteps,
                "multiway_speedup": cms / ms, "exact_match": True}

    # the partitioned plan on the same workload: R and S by H(B) into
    # shared-memory buckets (Algorithm 1 with the library's default bucket
    # count for row output)
    part = None
    if not args.no_partitioned and rank == 0:
        psh = ctx.plan_shares(binding.MWJ_LINEAR, dF, dF, dF, binding.MWJ_MATERIALIZE)
        rp = ctx.join3_linear(dF, dF, dF, "group_by_a", shares=psh, a_domain=a_domain)
        pexact = int(rp["total"].item()) == total and torch.equal(rp["counts"], r["counts"])
        pms = timed_ms(lambda: ctx.join3_linear(dF, dF, dF, "group_by_a", shares=psh, a_domain=a_domain,
                                                sync=False), stream, args.steps)
        part = {"impl": "partitioned: R and S by H(B), each bucket's B values in shared memory",
                "shares": list(psh), "value": 3 * n / (pms * 1e-3), "unit": UNIT, "ms_per_step": pms,
                "default_plan_speedup": pms / ms, "exact_match": bool(pexact)}

    star = None if args.no_star or rank != 0 else run_star(ctx, stream, args, peaks())
    skew = None if args.no_skew or rank != 0 else run_skew(ctx, stream, args)
    join4 = None if args.no_join4 or rank != 0 else run_join4(ctx, stream, args, F)
    fmr = None if args.no_fm or rank != 0 else run_fm(ctx, stream, args, F)

    # max over ranks
    if world > 1:
        ms, e2e_ms = max_over_ranks([ms, e2e_ms], dev)

    tuples = 3 * n
    value = replica_throughput(tuples, world, ms)
    peak, peak_kind = peaks()
    # T's single table and S's weight table: 2^k >= 4 x (estimated distinct
    # keys) slots of 8 bytes; both are keyed by F's source column here
    dc = int(np.count_nonzero(np.bincount(F[0], minlength=a_domain)))
    tslots = 16
    while tslots < 4 * dc:
        tslots *= 2
    wslots = tslots
    # dominant kernel and its roofline
    per_step = {k: v[0] / args.steps for k, v in phases.items()}
    dom = max(per_step, key=per_step.get) if per_step else None
    roof = None
    if dom:
        ab = algorithmic_bytes(dom, n, n, n, a_domain, tslots, phases[dom][1] / args.steps, wslots)
        if ab is not None:
            achieved = ab / (per_step[dom] * 1e-3) / 1e9
            tr = TRAFFIC.get(dom)
            traffic = (tr["bytes_per_step"] if tr and tr.get("digest") == source_digest(tr["sources"])
                       else None)
            roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                    "traffic": traffic, "peak_kind": peak_kind,
                    "algorithmic_bytes_per_step": ab,
                    "ms_per_step": round(per_step[dom], 4)}
    kernels = {k: {"ms_per_step": round(v[0] / args.steps, 4),
                   "launches_per_step": v[1] / args.steps} for k, v in phases.items()}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded power-law graph)",
        "config": {"workload": desc,
                   "impl": ("multiway (single-step 3-way hash join)" +
                            (", one bucket per side: T's table and S's weight table held in L2"
                             if tuple(shares[:2]) == (1, 1) else ", partitioned")),
                   "shares": list(shares), "tuples_per_step": tuples, "result_total": total,
                   "result_tuples_per_s": total * world / (ms * 1e-3),
                   "l2": "every input column pair (262 MB) exceeds the 129 MB L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof, "kernels": kernels,
        "e2e": {"value": replica_throughput(tuples, world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * a_domain + 8},
        "gpu_launches": launches, "clocks": clocks, "partitioned": part, "cascade": casc, "star": star,
        "skew": skew,
        "join4": join4, "fm": fmr,
    }
    return out, F


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

    def timed(fn, steps):
        for _ in range(3):
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

    r = ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=adom)
    # closed form: every fact tuple joins one tuple of each dimension
    inv = np.empty(nR, dtype=np.int64)
    inv[R[1]] = np.arange(nR)
    want = np.bincount(R[0][inv[S[0]]], minlength=adom)
    exact = int(r["total"].item()) == nS and np.array_equal(r["counts"].cpu().numpy(), want)
    ms = timed(lambda: ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=adom, sync=False), args.steps)
    ctx.set_profiling(True)
    ctx.reset_phase_times()
    for _ in range(args.steps):
        ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=adom, sync=False)
    torch.cuda.synchronize()
    ph = ctx.phase_times()
    ctx.set_profiling(False)
    probe_ms = ph.get("star_probe_groupby", (float("nan"), 0))[0] / args.steps
    # the probe reads S once (8 B per tuple) and both degree tables once
    slots = lambda n: 1 << max(4, int(np.ceil(np.log2(4 * n))))
    pbytes = 8 * nS + 8 * (slots(nR) + slots(nT))
    ach = pbytes / (probe_ms * 1e-3) / 1e9
    rc = ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=adom)
    exact = exact and torch.equal(rc["counts"], r["counts"])
    cms = timed(lambda: ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=adom,
                                         sync=False), max(3, args.steps // 4))
    return {"workload": f"star join: fact S(B,C) {nS} tuples (foreign keys, sorted by B), "
                        f"dimensions R(A,B), T(C,D) {nR} tuples each (unique keys), "
                        f"COUNT(*) GROUP BY A over 2^16 groups",
            "value": (nS + nR + nT) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "exact_match": bool(exact),
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
    import torch
    from paper_1905_13376_gb300 import binding, datagen

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
            "value": 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "exact_match": bool(exact),
            "result_total": int(want.sum()),
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
    for _ in range(3):
        ctx.join4_linear(dF, dF, dF, dF, "group_by_a", a_domain=adom, sync=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.join4_linear(dF, dF, dF, dF, "group_by_a", a_domain=adom, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
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
    for _ in range(3):
        ctx.fm_linear(dF, dF, dF, adom, sync=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.fm_linear(dF, dF, dF, adom, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    n = len(F[0])
    est = r["estimates"]
    return {"workload": "distinct friends of friends of friends per person, PCSA sketches "
                        "(16 x 32-bit bitmaps), F|x|F|x|F on the same graph",
            "value": 3 * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "median_estimate": float(est.median().item()), "max_estimate": float(est.max().item())}


def cpu_baseline(F, a_domain, budget_s=30.0):
    import oracle
    t0 = time.perf_counter()
    oracle.linear(F, F, F, oracle.GROUP_BY_A, a_domain=a_domain)
    dt = time.perf_counter() - t0
    n = len(F[0])
    return {"value": 3 * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the full workload once ({3 * n} input tuples, {dt:.2f} s, 1 thread)"}


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
            "config": {"workload": desc, "impl": "CPU oracle, single-threaded C hash join"},
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cascade", action="store_true")
    ap.add_argument("--no-partitioned", action="store_true",
                    help="skip timing the partitioned plan beside the default one")
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
    out, F = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(F, args.vertices)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
