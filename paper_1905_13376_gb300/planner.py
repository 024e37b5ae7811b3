"""The learned planner: choose the cascade or the 3-way join, and its share
vector, from a join instance's features.

A plan never changes a result, only its time.  Three plans are weighed:

  0  the cascade of binary hash joins (Section 6.3);
  1  the 3-way join with the library's default shares (linear: one bucket per
     side, both tables in L2; cyclic: R whole, C split into buckets);
  2  the 3-way join with the alternative shares of mwj_plan_shares_alt
     (linear: R and S by H(B) into shared-memory buckets; cyclic: the cube
     tiling of Section 5.2).

The network (24 -> 128 -> 128 -> 3, the library's BF16 kernels) predicts the
log2 microseconds of each plan and the planner takes the smallest; the
library's cost model (the paper's Appendix A restated for this GPU) is the
fallback and the yardstick of the learned planner's regret.

Training data is produced by the engine itself: seeded synthetic instances
are generated on the GPU, described by mwj_features, and every plan is timed
with CUDA events.  A cascade whose intermediate is estimated above
CASCADE_ROW_LIMIT rows is not run: its label is masked out of the training
loss and, in the evaluation, it counts as not runnable.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import binding

PLANS = ("cascade", "default", "alt")
CASCADE_ROW_LIMIT = 1 << 30       # larger intermediates are not run
REJECT_ROW_LIMIT = 1 << 33        # instances beyond this are not generated at all


# ---------------------------------------------------------------------------
# seeded instances on the GPU (data only: no join arithmetic)
# ---------------------------------------------------------------------------
_HTAB = {}


def _harmonic_gpu(s: float, device):
    import torch
    key = (round(s, 2), str(device))
    h = _HTAB.get(key)
    if h is None:
        k = torch.arange(1, (1 << 22) + 1, dtype=torch.float64, device=device)
        h = torch.cumsum(k.pow(-round(s, 2)), 0)
        _HTAB[key] = h
    return h


def gpu_column(gen, n: int, domain: int, zipf_s, device):
    import torch
    if zipf_s is None:
        return torch.randint(0, domain, (n,), generator=gen, device=device, dtype=torch.int64).to(torch.int32)
    H = _harmonic_gpu(zipf_s, device)[:domain]
    u = torch.rand(n, generator=gen, device=device, dtype=torch.float64) * H[-1]
    k = torch.searchsorted(H, u, right=True).clamp_(max=domain - 1)
    mult = int(torch.randint(1, max(2, domain), (1,), generator=gen, device=device).item())
    while math.gcd(mult, domain) != 1:
        mult = int(torch.randint(1, max(2, domain), (1,), generator=gen, device=device).item())
    off = int(torch.randint(0, domain, (1,), generator=gen, device=device).item())
    return ((k * mult + off) % domain).to(torch.int32)


@dataclass
class Instance:
    kind: int
    R: tuple
    S: tuple
    T: tuple
    sizes: tuple
    domains: tuple
    zipf_s: object


def gpu_instance(gen, rng: np.random.Generator, device, size_lo=1 << 10, size_hi=1 << 24,
                 dom_lo=1 << 6, dom_hi=1 << 22) -> Instance:
    kind = binding.MWJ_LINEAR if rng.random() < 0.5 else binding.MWJ_CYCLIC
    lu = lambda lo, hi: int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    nR, nS, nT = lu(size_lo, size_hi), lu(size_lo, size_hi), lu(size_lo, size_hi)
    s = float(rng.uniform(0.8, 1.5)) if rng.random() < 0.5 else None
    dA, dB, dC, dD = (lu(dom_lo, dom_hi) for _ in range(4))
    col = lambda n, d: gpu_column(gen, n, d, s, device)
    R = (col(nR, dA), col(nR, dB))
    S = (col(nS, dB), col(nS, dC))
    T = (col(nT, dC), col(nT, dD if kind == binding.MWJ_LINEAR else dA))
    return Instance(kind, R, S, T, (nR, nS, nT), (dA, dB, dC, dD), s)


# ---------------------------------------------------------------------------
# features, plans, timing
# ---------------------------------------------------------------------------
def features(ctx: binding.Context, kind, R, S, T) -> np.ndarray:
    import ctypes
    lib = ctx.lib
    ws = ctx.workspace(int(lib.mwj_features_workspace_size()))
    f = (ctypes.c_float * 24)()
    ctx._check(lib.mwj_features(ctx.h, kind, binding._rel(R), binding._rel(S), binding._rel(T), f,
                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctx._stream(None)))
    return np.array(f, dtype=np.float32)


def plan_shares(ctx, kind, R, S, T, plan: int):
    """Share vector of a 3-way plan (None: the library's default)."""
    if plan == 1:
        return None
    if plan == 2:
        return ctx.plan_shares_alt(kind, R, S, T)
    raise ValueError("the cascade has no shares")


def run_plan(ctx, kind, R, S, T, plan: int, mode="count", **kw):
    if plan == 0:
        return ctx.cascade_join(kind, R, S, T, mode, **kw)
    sh = plan_shares(ctx, kind, R, S, T, plan)
    if kind == binding.MWJ_LINEAR:
        return ctx.join3_linear(R, S, T, mode, shares=sh, **kw)
    return ctx.join3_cyclic(R, S, T, mode, shares=sh, **kw)


def time_plan(ctx, inst: Instance, plan: int, reps: int = 2, rows_hint: float = 0):
    import torch
    kw = {}
    if plan == 0:   # room for the whole intermediate when it is known to be large
        per_row = 12 if inst.kind == binding.MWJ_LINEAR else 20
        kw["workspace_bytes"] = int(min(2.0 * rows_hint, 2.0 ** 31) * per_row) + (256 << 20)
    r = run_plan(ctx, inst.kind, inst.R, inst.S, inst.T, plan, **kw)   # warm-up, synchronised
    total = int(r["total"].item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run_plan(ctx, inst.kind, inst.R, inst.S, inst.T, plan, sync=False, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps, total


def measure(ctx, inst: Instance, f: np.ndarray):
    """Times (us) of the three plans (None: not run) and the join's total;
    every plan that runs must give the same total."""
    rows_est = 2.0 ** float(f[8]) - 1.0
    t = [None, None, None]
    totals = set()
    for p in (1, 2):
        t[p], tot = time_plan(ctx, inst, p)
        totals.add(tot)
    if rows_est <= CASCADE_ROW_LIMIT:
        t[0], tot = time_plan(ctx, inst, 0, rows_hint=rows_est)
        totals.add(tot)
    if len(totals) != 1:
        raise AssertionError(f"plans disagree on the result: {sorted(totals)}")
    return t, totals.pop()


# ---------------------------------------------------------------------------
# the planner
# ---------------------------------------------------------------------------
class Planner:
    """Normalisation + network; choose() returns the plan index (0, 1, 2)."""

    def __init__(self, ctx, params=None, fmean=None, fstd=None, ymean=None, ystd=None):
        self.ctx = ctx
        self.mlp = binding.MLP(ctx, params)
        self.fmean = np.zeros(24, np.float32) if fmean is None else np.asarray(fmean, np.float32)
        self.fstd = np.ones(24, np.float32) if fstd is None else np.asarray(fstd, np.float32)
        self.ymean = np.zeros(3, np.float32) if ymean is None else np.asarray(ymean, np.float32)
        self.ystd = np.ones(3, np.float32) if ystd is None else np.asarray(ystd, np.float32)

    def predict(self, F: np.ndarray) -> np.ndarray:
        """Predicted log2 microseconds of the three plans, one row per instance."""
        import torch
        X = torch.from_numpy(((F - self.fmean) / self.fstd).astype(np.float32)).to(self.ctx.device)
        Y = self.mlp.forward(X).cpu().numpy()
        return Y * self.ystd + self.ymean

    def choose(self, F: np.ndarray):
        return [int(np.argmin(p)) for p in self.predict(np.atleast_2d(F))]

    def save(self, path):
        np.savez(path, params=self.mlp.get_params(), fmean=self.fmean, fstd=self.fstd,
                 ymean=self.ymean, ystd=self.ystd)

    @classmethod
    def load(cls, ctx, path):
        d = np.load(path)
        return cls(ctx, d["params"], d["fmean"], d["fstd"], d["ymean"], d["ystd"])


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "planner_weights.npz")


def default_planner(ctx) -> Planner:
    """The network trained on engine-timed instances (planner_weights.npz)."""
    return Planner.load(ctx, WEIGHTS)


def cost_model_choice(F: np.ndarray, hbm_gbs=6792.1):
    return [int(np.argmin(binding.cost_model(f, hbm_gbs))) for f in np.atleast_2d(F)]


def runnable(choice: int, f: np.ndarray) -> int:
    """The plan that runs for a choice: the 3-way join with the default shares
    instead of a cascade whose estimated intermediate would not fit."""
    if choice == 0 and 2.0 ** float(f[8]) - 1.0 > CASCADE_ROW_LIMIT:
        return 1
    return choice


def plan_and_run(ctx, kind, R, S, T, mode="count", planner: Planner | None = None, **kw):
    """Choose a plan (the learned planner, else the cost model) and run it.
    Returns (result, plan index)."""
    F = features(ctx, kind, R, S, T)
    choice = runnable((planner.choose(F) if planner is not None else cost_model_choice(F))[0], F)
    return run_plan(ctx, kind, R, S, T, choice, mode, **kw), choice


def labels(times):
    """Targets log2 us of the three plans; mask 0 where a plan was not run."""
    Y = np.zeros((len(times), 3), np.float32)
    M = np.zeros((len(times), 3), np.float32)
    for i, t in enumerate(times):
        for p in range(3):
            if t[p] is not None:
                Y[i, p] = math.log2(max(t[p], 1e-3))
                M[i, p] = 1.0
    return Y, M


def plan_time(t, p):
    return t[p] if t[p] is not None else float("inf")


def train(planner: Planner, F, Y, M, steps=3000, batch=512, lr=1e-3, seed=0, log=None):
    import torch
    planner.fmean = F.mean(0)
    planner.fstd = F.std(0) + 1e-3
    planner.ymean = (Y * M).sum(0) / np.maximum(M.sum(0), 1)
    planner.ystd = np.sqrt(((Y - planner.ymean) ** 2 * M).sum(0) / np.maximum(M.sum(0), 1)) + 1e-3
    dev = planner.ctx.device
    X = torch.from_numpy(((F - planner.fmean) / planner.fstd).astype(np.float32)).to(dev)
    T = torch.from_numpy(((Y - planner.ymean) / planner.ystd).astype(np.float32)).to(dev)
    Mt = torch.from_numpy(M.astype(np.float32)).to(dev)
    g = np.random.default_rng(seed)
    losses = []
    for step in range(steps):
        idx = torch.from_numpy(g.choice(len(F), min(batch, len(F)), replace=False)).to(dev)
        _, loss = planner.mlp.backward(X[idx], T[idx], Mt[idx])
        planner.mlp.adam(lr * (0.1 if step > 0.8 * steps else 1.0))
        if step % 200 == 0 or step == steps - 1:
            losses.append((step, float(loss.item())))
            if log:
                log(f"step {step} loss {losses[-1][1]:.4f}")
    return losses


def evaluate(planner: Planner, F, times, sizes=None):
    """Regret t(plan) / t(best measured plan) - 1 of the learned planner, the
    cost model alone (each choice as plan_and_run runs it), and each fixed
    plan, on instances whose 3-way plans were all timed; and, where the
    intermediate |R join S| exceeds the inputs |R| + |S| + |T|, the learned
    plan's speed-up over the plain cascade."""
    learned = [runnable(c, f) for c, f in zip(planner.choose(F), np.atleast_2d(F))]
    model = [runnable(c, f) for c, f in zip(cost_model_choice(F), np.atleast_2d(F))]
    res = {"learned": [], "cost_model": [], "cascade": [], "default": [], "alt": []}
    big_speedup, big_beats = [], []
    for i, t in enumerate(times):
        b = min(plan_time(t, p) for p in range(3))
        res["learned"].append(plan_time(t, learned[i]) / b - 1)
        res["cost_model"].append(plan_time(t, model[i]) / b - 1)
        for p, name in enumerate(PLANS):
            res[name].append(plan_time(t, p) / b - 1)
        inputs = (sum(sizes[i]) if sizes is not None else
                  sum(2.0 ** float(F[i][k]) - 1.0 for k in range(3)))
        if 2.0 ** float(F[i][8]) - 1.0 > inputs:
            tc = plan_time(t, 0)
            tl = plan_time(t, learned[i])
            big_speedup.append(tc / tl)
            big_beats.append(tl < tc)
    summary = {}
    for k, v in res.items():
        a = np.array(v)
        fin = np.isfinite(a)
        summary[k] = {"mean_regret": float(np.mean(a[fin])) if fin.any() else None,
                      "geo_mean_slowdown": float(np.exp(np.mean(np.log1p(a[fin])))) if fin.any() else None,
                      "within_10pct": float(np.mean(a <= 0.10)),
                      "not_runnable": int((~fin).sum())}
    bs = np.array(big_speedup)
    fin = np.isfinite(bs)
    summary["intermediate_above_inputs"] = {
        "instances": len(big_speedup),
        "learned_beats_cascade": float(np.mean(big_beats)) if big_beats else None,
        "geo_mean_speedup_over_cascade_runnable": float(np.exp(np.mean(np.log(bs[fin])))) if fin.any() else None,
        "cascade_not_runnable": int((~fin).sum())}
    summary["n"] = len(times)
    return summary, res


# ---------------------------------------------------------------------------
# data collection and the training run
# ---------------------------------------------------------------------------
def collect(ctx, n: int, seed: int, budget_s: float, log=None, keep_small: int = 0, **kw):
    """Up to n timed instances (stops early when budget_s seconds are spent).
    Returns features, times, totals, metadata and the count of instances
    rejected (intermediate above REJECT_ROW_LIMIT, or a workspace the GPU
    cannot hold).  With keep_small > 0 each metadata entry of an instance of
    at most keep_small tuples in all also holds host copies of its relations
    ("rel"), so that its total can be checked elsewhere."""
    import torch
    gen = torch.Generator(device=ctx.device)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    F, times, totals, meta = [], [], [], []
    t0 = time.time()
    rejected = 0
    while len(F) < n and time.time() - t0 < budget_s:
        inst = gpu_instance(gen, rng, ctx.device, **kw)
        f = features(ctx, inst.kind, inst.R, inst.S, inst.T)
        if 2.0 ** float(f[8]) > REJECT_ROW_LIMIT:
            rejected += 1
            continue
        try:
            t, tot = measure(ctx, inst, f)
        except binding.MwjError as e:
            if e.status == binding.MWJ_ERR_WORKSPACE:
                rejected += 1
                continue
            raise
        except torch.cuda.OutOfMemoryError:
            ctx._ws = None
            torch.cuda.empty_cache()
            rejected += 1
            continue
        F.append(f)
        times.append(t)
        totals.append(tot)
        m = {"kind": int(inst.kind), "sizes": list(inst.sizes), "domains": list(inst.domains),
             "zipf": inst.zipf_s}
        if keep_small and sum(inst.sizes) <= keep_small:
            m["rel"] = [tuple(c.cpu().numpy() for c in rel) for rel in (inst.R, inst.S, inst.T)]
        meta.append(m)
        if log and len(F) % 1000 == 0:
            log(f"{len(F)} instances, {time.time() - t0:.0f} s, rejected {rejected}")
    return np.array(F, np.float32), times, totals, meta, rejected


def _times_to_array(times):
    A = np.full((len(times), 3), np.nan)
    for i, t in enumerate(times):
        for p in range(3):
            if t[p] is not None:
                A[i, p] = t[p]
    return A


def _array_to_times(A):
    return [[None if np.isnan(v) else float(v) for v in row] for row in A]


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--eval", type=int, default=512)
    ap.add_argument("--budget", type=float, default=1200.0, help="seconds for collecting training data")
    ap.add_argument("--size-hi", type=int, default=1 << 24)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--out", default="planner_run")
    ap.add_argument("--seed", type=int, default=1905)
    ap.add_argument("--eval-only", action="store_true",
                    help="time held-out instances on this engine and score the packaged weights")
    ap.add_argument("--from-dataset", default=None,
                    help="train and score from a saved dataset.npz (+ meta.json beside it) without timing again")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    log = lambda m: print(m, flush=True)
    torch.cuda.set_device(0)
    ctx = binding.Context(0)
    t0 = time.time()
    if args.eval_only:
        Fev, tev, _, mev, rej2 = collect(ctx, args.eval, args.seed + 1, 1e9, log, size_hi=args.size_hi)
        summary, _ = evaluate(default_planner(ctx), Fev, tev, [m["sizes"] for m in mev])
        rep = {"n_eval": len(Fev), "rejected": rej2, "eval": summary, "collect_seconds": time.time() - t0,
               "weights": "packaged planner_weights.npz"}
        json.dump(rep, open(os.path.join(args.out, "report_eval.json"), "w"), indent=1)
        log(json.dumps(rep, indent=1))
        return
    if args.from_dataset:
        d = np.load(args.from_dataset)
        meta = json.load(open(os.path.join(os.path.dirname(args.from_dataset), "meta.json")))
        Ftr, ttr, Fev, tev = d["Ftrain"], _array_to_times(d["Ttrain"]), d["Feval"], _array_to_times(d["Teval"])
        mtr, mev, rej, rej2 = meta["train_meta"], meta["eval_meta"], None, None
        log(f"dataset {args.from_dataset}: {len(Ftr)} training and {len(Fev)} held-out instances")
    else:
        Ftr, ttr, _, mtr, rej = collect(ctx, args.train, args.seed, args.budget, log, size_hi=args.size_hi)
        log(f"train: {len(Ftr)} instances in {time.time() - t0:.0f} s ({rej} rejected)")
        Fev, tev, totev, mev, rej2 = collect(ctx, args.eval, args.seed + 1, 1e9, log, size_hi=args.size_hi)
        np.savez(os.path.join(args.out, "dataset.npz"), Ftrain=Ftr, Ttrain=_times_to_array(ttr),
                 Feval=Fev, Teval=_times_to_array(tev), totals_eval=np.array(totev, dtype=np.int64))
        json.dump({"train_meta": mtr, "eval_meta": mev}, open(os.path.join(args.out, "meta.json"), "w"))
    Y, M = labels(ttr)
    planner = Planner(ctx, _init(args.seed))
    losses = train(planner, Ftr, Y, M, steps=args.steps, log=log)
    planner.save(os.path.join(args.out, "planner.npz"))
    summary, _ = evaluate(planner, Fev, tev, [m["sizes"] for m in mev])
    rep = {"n_train": len(Ftr), "n_eval": len(Fev), "rejected_train": rej, "rejected_eval": rej2,
           "size_hi": args.size_hi, "losses": losses, "eval": summary, "collect_seconds": time.time() - t0}
    json.dump(rep, open(os.path.join(args.out, "report.json"), "w"), indent=1)
    log(json.dumps(rep["eval"], indent=1))


def _init(seed: int):
    """He-uniform weights, zero biases (the network's initial point)."""
    g = np.random.default_rng(seed)
    parts = []
    for shape in [(24, 128), (128,), (128, 128), (128,), (128, 3), (3,)]:
        if len(shape) == 2:
            lim = math.sqrt(6.0 / shape[0])
            parts.append(g.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


if __name__ == "__main__":
    main()
