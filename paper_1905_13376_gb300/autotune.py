"""Autotuner of batched joins.

A batch of independent 3-way joins (mwj_batch_*) plans every query from its
sizes with a rule: about `tuples_per_bucket` R tuples per H(B) bucket and a
T degree table of `table_factor` slots per tuple for linear queries, and the
cube shares of Section 5.2's z|R| + x|S| + y|T| searched with R_ij and T_ki
filling at most `fit_pct` % of a tile's on-chip capacity for cyclic ones.
The batch then runs in one persistent partitioning launch and one persistent
join launch, each with a number of CTAs per SM.

autotune() picks these per (kind, size class) -- size class
floor(log2(max(|R|, |S|, |T|))) -- and the two launch shapes by timing the
candidates on the engine with the caller's own queries (a sample of each
class, a batch of that sample per candidate), keeps a candidate only when it
beats the library's rule by more than the timing noise, and installs the
result in the context (mwj_batch_set_rules / mwj_batch_set_launch).  The
result is a plain dict that save() and load() keep as JSON, so that a later
process installs it without tuning again.  Rules change plans only, never a
count.
"""
from __future__ import annotations

import json
import math
import time
from collections import defaultdict

import numpy as np

from . import binding

LINEAR_TPB = (2048, 4096, 8192, 16384, 32768)
LINEAR_TFAC = (2, 4)
CYCLIC_FIT = (25, 35, 50, 65, 80)
LAUNCH = ((0, 0), (2, 0), (4, 0), (3, 1), (3, 2))
DEFAULT = {binding.MWJ_LINEAR: (8192, 2, 0), binding.MWJ_CYCLIC: (0, 0, 50)}
MARGIN = 0.03   # a candidate must beat the library's rule by this fraction


def size_class(R, S, T) -> int:
    m = max(R[0].numel(), S[0].numel(), T[0].numel(), 1)
    return int(math.floor(math.log2(m)))


def _rule_list(rules: dict):
    return [(k, c, tpb, tfac, fit) for (k, c), (tpb, tfac, fit) in sorted(rules.items())]


def _time_batch(ctx, queries, reps: int) -> float:
    """Milliseconds of one launch of a batch of `queries` (after the launch
    that binds its workspace), mean of `reps`."""
    import torch
    b = binding.Batch(ctx, queries)
    try:
        b.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.launch()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        b.close()


def autotune(ctx: binding.Context, queries, sample: int = 32, reps: int = 3, seed: int = 0, log=None) -> dict:
    """Tune the batch rules and launch shapes on `queries` (a list of
    (kind, R, S, T) with device relations whose shares the library chooses).
    Installs the result in ctx and returns it."""
    t0 = time.time()
    groups = defaultdict(list)
    for i, q in enumerate(queries):
        groups[(int(q[0]), size_class(*q[1:4]))].append(i)
    rng = np.random.default_rng(seed)
    rules, timings = {}, {}
    ctx.batch_set_rules([])
    ctx.batch_set_launch(0, 0)
    for key in sorted(groups):
        idx = groups[key]
        pick = idx if len(idx) <= sample else sorted(rng.choice(idx, sample, replace=False).tolist())
        sub = [queries[i][:4] for i in pick]
        kind, _ = key
        cands = ([(t, f, 0) for t in LINEAR_TPB for f in LINEAR_TFAC] if kind == binding.MWJ_LINEAR
                 else [(0, 0, fit) for fit in CYCLIC_FIT])
        base = DEFAULT[kind]
        res = {}
        for c in [base] + [c for c in cands if c != base]:
            trial = dict(rules)
            trial[key] = c
            ctx.batch_set_rules(_rule_list(trial))
            res[c] = _time_batch(ctx, sub, reps)
        best = min(res, key=res.get)
        if res[best] > (1.0 - MARGIN) * res[base]:
            best = base
        rules[key] = best
        timings[f"{kind}:{key[1]}"] = {"queries": len(sub), "default_ms": res[base], "best_ms": res[best],
                                       "best": list(best)}
        if log:
            log(f"class {key}: {len(sub)} queries, {res[base]:.3f} -> {res[best]:.3f} ms with {best}")
    ctx.batch_set_rules(_rule_list(rules))
    # the launch shapes, on a sample of the whole batch
    n_all = len(queries)
    pick = list(range(n_all)) if n_all <= 8 * sample else sorted(
        rng.choice(n_all, 8 * sample, replace=False).tolist())
    sub = [queries[i][:4] for i in pick]
    lres = {}
    for lp in LAUNCH:
        ctx.batch_set_launch(*lp)
        lres[lp] = _time_batch(ctx, sub, reps)
    launch = min(lres, key=lres.get)
    if lres[launch] > (1.0 - MARGIN) * lres[(0, 0)]:
        launch = (0, 0)
    ctx.batch_set_launch(*launch)
    return {"rules": [list(r) for r in _rule_list(rules)], "launch": list(launch),
            "class_timings": timings, "launch_timings_ms": {f"{a},{b}": v for (a, b), v in lres.items()},
            "tuning_seconds": time.time() - t0}


def install(ctx: binding.Context, tuning: dict):
    ctx.batch_set_rules([tuple(r) for r in tuning["rules"]])
    ctx.batch_set_launch(*tuning["launch"])


def save(tuning: dict, path: str):
    with open(path, "w") as fh:
        json.dump(tuning, fh, indent=1)


def load(path: str) -> dict:
    with open(path) as fh:
        return json.load(fh)
