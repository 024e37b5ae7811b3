"""The learned planner: choose the cascade or the 3-way join, and scale the
shares, from a join instance's features.

A plan never changes a result, only its time.  The network (24 -> 128 ->
128 -> 3, the library's BF16 kernels) predicts log2 microseconds of the
cascade, log2 microseconds of the 3-way join with the default shares, and
the best share scale k (shares x 2^k, k in {-1, 0, 1}); the cost model of
the library is the fallback and the yardstick of the learned planner's
regret.

Training data is produced by the engine itself: seeded synthetic instances
are generated on the GPU, described by mwj_features, and every plan is timed
with CUDA events.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import binding

SCALES = (-1, 0, 1)
CASCADE_ROW_LIMIT = 1 << 30       # larger intermediates are not run (labelled by the model)
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


def gpu_instance(gen, rng: np.random.Generator, device, size_lo=1 << 10, size_hi=1 << 22,
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


def scaled_shares(ctx, kind, R, S, T, k: int):
    # the scale applies to the partitioned plan (the library's default for
    # row output); the one-bucket plan the linear aggregates default to is
    # not in this family
    base = ctx.plan_shares(kind, R, S, T, binding.MWJ_MATERIALIZE)
    if kind == binding.MWJ_LINEAR:
        I = max(1, min(16384, int(base[0] * 2.0 ** k)))
        return (I, 1, 1)
    sh = [max(1, int(v * 2.0 ** k)) for v in base]
    while sh[0] * sh[1] > 32768 or sh[1] * sh[2] > 32768 or sh[2] * sh[0] > 32768:
        sh = [max(1, v // 2) for v in sh]
    return tuple(sh)


def run_plan(ctx, kind, R, S, T, cascade: bool, k: int = 0, mode="count", **kw):
    if cascade:
        return ctx.cascade_join(kind, R, S, T, mode, **kw)
    sh = scaled_shares(ctx, kind, R, S, T, k)
    if kind == binding.MWJ_LINEAR:
        return ctx.join3_linear(R, S, T, mode, shares=sh, **kw)
    return ctx.join3_cyclic(R, S, T, mode, shares=sh, **kw)


def time_plan(ctx, inst: Instance, cascade: bool, k: int = 0, reps: int = 1, rows_hint: float = 0):
    import torch
    kw = {}
    if cascade:   # room for the whole intermediate when it is known to be large
        per_row = 12 if inst.kind == binding.MWJ_LINEAR else 20
        kw["workspace_bytes"] = int(min(2.0 * rows_hint, 2.0 ** 31) * per_row) + (256 << 20)
    run_plan(ctx, inst.kind, inst.R, inst.S, inst.T, cascade, k, **kw)   # warm-up, synchronised
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        r = run_plan(ctx, inst.kind, inst.R, inst.S, inst.T, cascade, k, sync=False, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps, int(r["total"].item())


def measure(ctx, inst: Instance, f: np.ndarray):
    """Times (us) of the cascade and of the 3-way join at every share scale."""
    rows_est = 2.0 ** float(f[8]) - 1.0
    t = {}
    totals = set()
    for k in SCALES:
        t[("mw", k)], tot = time_plan(ctx, inst, False, k)
        totals.add(tot)
    if rows_est <= CASCADE_ROW_LIMIT:
        t["cascade"], tot = time_plan(ctx, inst, True, rows_hint=rows_est)
        totals.add(tot)
    else:
        t["cascade"] = None
    if len(totals) != 1:
        raise AssertionError(f"plans disagree on the result: {sorted(totals)}")
    return t, totals.pop()


# ---------------------------------------------------------------------------
# the planner
# ---------------------------------------------------------------------------
class Planner:
    """Normalisation + network; choose() returns (cascade?, share scale)."""

    def __init__(self, ctx, params=None, fmean=None, fstd=None, ymean=None, ystd=None):
        self.ctx = ctx
        self.mlp = binding.MLP(ctx, params)
        self.fmean = np.zeros(24, np.float32) if fmean is None else np.asarray(fmean, np.float32)
        self.fstd = np.ones(24, np.float32) if fstd is None else np.asarray(fstd, np.float32)
        self.ymean = np.zeros(3, np.float32) if ymean is None else np.asarray(ymean, np.float32)
        self.ystd = np.ones(3, np.float32) if ystd is None else np.asarray(ystd, np.float32)

    def predict(self, F: np.ndarray) -> np.ndarray:
        import torch
        X = torch.from_numpy(((F - self.fmean) / self.fstd).astype(np.float32)).to(self.ctx.device)
        Y = self.mlp.forward(X).cpu().numpy()
        return Y * self.ystd + self.ymean

    def choose(self, F: np.ndarray):
        P = self.predict(np.atleast_2d(F))
        return [(bool(p[0] < p[1]), int(np.clip(np.rint(p[2]), -1, 1))) for p in P]

    def save(self, path):
        np.savez(path, params=self.mlp.get_params(), fmean=self.fmean, fstd=self.fstd,
                 ymean=self.ymean, ystd=self.ystd)

    @classmethod
    def load(cls, ctx, path):
        d = np.load(path)
        return cls(ctx, d["params"], d["fmean"], d["fstd"], d["ymean"], d["ystd"])


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "planner_weights.npz")


def default_planner(ctx) -> Planner:
    """The network trained on 20000 engine-timed instances (planner_weights.npz)."""
    return Planner.load(ctx, WEIGHTS)


def plan_and_run(ctx, kind, R, S, T, mode="count", planner: Planner | None = None, **kw):
    """Choose a plan (the learned planner, else the cost model) and run it.
    Returns (result, (cascade?, share scale))."""
    F = features(ctx, kind, R, S, T)
    choice = (planner.choose(F) if planner is not None else cost_model_choice(F))[0]
    return run_plan(ctx, kind, R, S, T, choice[0], choice[1], mode, **kw), choice


def cost_model_choice(F: np.ndarray, hbm_gbs=6792.1):
    out = []
    for f in np.atleast_2d(F):
        c = binding.cost_model(f, hbm_gbs)
        out.append((bool(c[0] < c[1]), int(np.rint(c[2]))))
    return out


def labels(times, F, calib):
    """Targets: log2 us of the cascade, of the 3-way join (scale 0), best scale."""
    Y = np.zeros((len(times), 3), np.float32)
    M = np.ones((len(times), 3), np.float32)
    for i, t in enumerate(times):
        tc = t["cascade"]
        if tc is None:   # not run: the cost model's prediction, calibrated on the runs
            tc = 2.0 ** (binding.cost_model(F[i])[0] + calib) * 1e6
        Y[i, 0] = math.log2(tc)
        Y[i, 1] = math.log2(t[("mw", 0)])
        Y[i, 2] = min(SCALES, key=lambda k: t[("mw", k)])
    return Y, M


def calibration(times, F):
    d = [math.log2(t["cascade"] * 1e-6) - binding.cost_model(F[i])[0]
         for i, t in enumerate(times) if t["cascade"] is not None]
    return float(np.median(d)) if d else 0.0


def plan_time(t, choice):
    cascade, k = choice
    if cascade:
        return t["cascade"] if t["cascade"] is not None else float("inf")
    return t[("mw", k)]


def best_time(t):
    c = [v for key, v in t.items() if v is not None]
    return min(c)


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


def evaluate(planner: Planner, F, times):
    """Regret t(plan)/t(best) - 1 of the learned planner, the cost model and
    the plain cascade on instances whose plans were all timed."""
    learned = planner.choose(F)
    model = cost_model_choice(F)
    res = {"learned": [], "cost_model": [], "cascade": [], "multiway_default": []}
    for i, t in enumerate(times):
        b = best_time(t)
        res["learned"].append(plan_time(t, learned[i]) / b - 1)
        res["cost_model"].append(plan_time(t, model[i]) / b - 1)
        res["cascade"].append(plan_time(t, (True, 0)) / b - 1)
        res["multiway_default"].append(plan_time(t, (False, 0)) / b - 1)
    summary = {}
    for k, v in res.items():
        a = np.array(v)
        fin = np.isfinite(a)
        summary[k] = {"mean_regret": float(np.mean(np.where(fin, a, np.nan)[fin])) if fin.any() else None,
                      "geo_mean_slowdown": float(np.exp(np.mean(np.log1p(a[fin])))) if fin.any() else None,
                      "within_10pct": float(np.mean(a <= 0.10)),
                      "not_runnable": int((~fin).sum())}
    return summary, res


# ---------------------------------------------------------------------------
# data collection and the training run
# ---------------------------------------------------------------------------
def collect(ctx, n: int, seed: int, budget_s: float, log=None, **kw):
    """Up to n timed instances (stops early when budget_s seconds are spent)."""
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
        F.append(f)
        times.append(t)
        totals.append(tot)
        meta.append({"kind": int(inst.kind), "sizes": list(inst.sizes), "domains": list(inst.domains),
                     "zipf": inst.zipf_s})
        if log and len(F) % 500 == 0:
            log(f"{len(F)} instances, {time.time() - t0:.0f} s, rejected {rejected}")
    return np.array(F, np.float32), times, totals, meta, rejected


def _times_to_arrays(times):
    keys = ["cascade"] + [("mw", k) for k in SCALES]
    A = np.full((len(times), len(keys)), np.nan)
    for i, t in enumerate(times):
        for j, k in enumerate(keys):
            if t[k] is not None:
                A[i, j] = t[k]
    return A


def _arrays_to_times(A):
    keys = ["cascade"] + [("mw", k) for k in SCALES]
    out = []
    for row in A:
        out.append({k: (None if np.isnan(row[j]) else float(row[j])) for j, k in enumerate(keys)})
    return out


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--eval", type=int, default=512)
    ap.add_argument("--budget", type=float, default=900.0, help="seconds for collecting training data")
    ap.add_argument("--size-hi", type=int, default=1 << 22)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--out", default="planner_run")
    ap.add_argument("--seed", type=int, default=1905)
    ap.add_argument("--eval-only", action="store_true",
                    help="time the held-out instances on this engine and score the packaged weights")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    log = lambda m: print(m, flush=True)
    torch.cuda.set_device(0)
    ctx = binding.Context(0)
    t0 = time.time()
    if args.eval_only:
        Fev, tev, totev, mev, rej2 = collect(ctx, args.eval, args.seed + 1, 1e9, log, size_hi=args.size_hi)
        summary, _ = evaluate(default_planner(ctx), Fev, tev)
        rep = {"n_eval": len(Fev), "eval": summary, "collect_seconds": time.time() - t0,
               "weights": "packaged planner_weights.npz"}
        json.dump(rep, open(os.path.join(args.out, "report_eval.json"), "w"), indent=1)
        log(json.dumps(rep, indent=1))
        return
    Ftr, ttr, _, mtr, rej = collect(ctx, args.train, args.seed, args.budget, log, size_hi=args.size_hi)
    log(f"train: {len(Ftr)} instances in {time.time() - t0:.0f} s ({rej} rejected)")
    Fev, tev, totev, mev, rej2 = collect(ctx, args.eval, args.seed + 1, 1e9, log, size_hi=args.size_hi)
    np.savez(os.path.join(args.out, "dataset.npz"), Ftrain=Ftr, Ttrain=_times_to_arrays(ttr),
             Feval=Fev, Teval=_times_to_arrays(tev), totals_eval=np.array(totev, dtype=np.int64))
    json.dump({"train_meta": mtr, "eval_meta": mev}, open(os.path.join(args.out, "meta.json"), "w"))
    calib = calibration(ttr, Ftr)
    Y, M = labels(ttr, Ftr, calib)
    planner = Planner(ctx, _init(args.seed))
    losses = train(planner, Ftr, Y, M, steps=args.steps, log=log)
    planner.save(os.path.join(args.out, "planner.npz"))
    summary, _ = evaluate(planner, Fev, tev)
    rep = {"n_train": len(Ftr), "n_eval": len(Fev), "calibration_log2": calib, "losses": losses,
           "eval": summary, "collect_seconds": time.time() - t0}
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
