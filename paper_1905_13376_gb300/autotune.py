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
candidates on the engine with the caller's own queries (inside a sample of
the whole batch, so that each candidate shares the launches with the rest of
the mix), keeps a candidate only when it beats the current choice by more
than the timing noise and the result only when it beats the library's rule
on the whole batch, and installs the result in the context
(mwj_batch_set_rules / mwj_batch_set_launch).  The
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


def _tuples(q) -> int:
    return sum(int(c.numel()) for rel in q[1:4] for c in rel[:1])


def autotune(ctx: binding.Context, queries, context: int = 1024, reps: int = 3, seed: int = 0,
             log=None) -> dict:
    """Tune the batch rules and launch shapes on `queries` (a list of
    (kind, R, S, T) with device relations whose shares the library chooses).

    A query's plan changes how the batch's two persistent launches share
    their CTAs with every other query, so candidates are timed inside a
    batch of the caller's mix: a sample of `context` queries, in which one
    class's rule is varied at a time (classes with the most tuples first)
    and kept when the sample's launch gets faster by more than MARGIN.  The
    result is then timed on the whole batch against the library's rule and
    kept only if it wins there as well.  Installs the result in ctx and
    returns it."""
    t0 = time.time()
    groups = defaultdict(list)
    for i, q in enumerate(queries):
        groups[(int(q[0]), size_class(*q[1:4]))].append(i)
    rng = np.random.default_rng(seed)
    n_all = len(queries)
    pick = list(range(n_all)) if n_all <= context else sorted(rng.choice(n_all, context, replace=False).tolist())
    sub = [queries[i][:4] for i in pick]
    in_sub = set(pick)
    weight = {key: sum(_tuples(queries[i]) for i in idx if i in in_sub) for key, idx in groups.items()}
    ctx.batch_set_rules([])
    ctx.batch_set_launch(0, 0)
    cur = _time_batch(ctx, sub, reps)
    rules, timings = {}, {}
    for key in sorted(groups, key=lambda k: -weight[k]):
        if weight[key] == 0:
            continue
        kind, _ = key
        cands = ([(t, f, 0) for t in LINEAR_TPB for f in LINEAR_TFAC] if kind == binding.MWJ_LINEAR
                 else [(0, 0, fit) for fit in CYCLIC_FIT])
        base = DEFAULT[kind]
        res = {base: cur}
        for c in cands:
            if c == base:
                continue
            trial = dict(rules)
            trial[key] = c
            ctx.batch_set_rules(_rule_list(trial))
            res[c] = _time_batch(ctx, sub, reps)
        best = min(res, key=res.get)
        if best != base and res[best] < (1.0 - MARGIN) * cur:
            rules[key] = best
            cur = res[best]
        ctx.batch_set_rules(_rule_list(rules))
        timings[f"{kind}:{key[1]}"] = {"queries": len(groups[key]), "context_ms_before": res[base],
                                       "context_ms_after": cur, "rule": list(rules.get(key, base))}
        if log:
            log(f"class {key}: {res[base]:.3f} -> {cur:.3f} ms with {rules.get(key, base)}")
    # the launch shapes, in the same sample
    lres = {(0, 0): cur}
    for lp in LAUNCH:
        if lp != (0, 0):
            ctx.batch_set_launch(*lp)
            lres[lp] = _time_batch(ctx, sub, reps)
    launch = min(lres, key=lres.get)
    if lres[launch] > (1.0 - MARGIN) * lres[(0, 0)]:
        launch = (0, 0)
    # the whole batch: tuned against the library's rule
    full = [q[:4] for q in queries]
    ctx.batch_set_launch(*launch)
    tuned_ms = _time_batch(ctx, full, reps)
    ctx.batch_set_rules([])
    ctx.batch_set_launch(0, 0)
    library_ms = _time_batch(ctx, full, reps)
    kept = tuned_ms < (1.0 - MARGIN) * library_ms
    if not kept:
        rules, launch = {}, (0, 0)
    ctx.batch_set_rules(_rule_list(rules))
    ctx.batch_set_launch(*launch)
    return {"rules": [list(r) for r in _rule_list(rules)], "launch": list(launch),
            "class_timings": timings, "launch_timings_ms": {f"{a},{b}": v for (a, b), v in lres.items()},
            "whole_batch_ms": {"tuned": tuned_ms, "library_rule": library_ms, "kept": bool(kept)},
            "context_queries": len(sub), "tuning_seconds": time.time() - t0}


def install(ctx: binding.Context, tuning: dict):
    ctx.batch_set_rules([tuple(r) for r in tuning["rules"]])
    ctx.batch_set_launch(*tuning["launch"])


def save(tuning: dict, path: str):
    with open(path, "w") as fh:
        json.dump(tuning, fh, indent=1)


def load(path: str) -> dict:
    with open(path) as fh:
        return json.load(fh)
