"""The planner's pieces on the GPU: BF16 network forward/backward against the
CPU oracle, training, features against exact values, and what the trained
network gains over the cost model alone."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1905_13376_gb300 import binding, datagen, planner

from gpu_util import cu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.set_device(0)
    c = binding.Context(0)
    yield c
    c.close()


def _params(seed):
    g = np.random.default_rng(seed)
    p = omlp.init_params(seed).astype(np.float64)
    p += g.normal(0, 0.02, p.size)       # nonzero biases too
    return p.astype(np.float32)


def test_mlp_forward_matches_oracle(ctx):
    import torch
    p = _params(1)
    net = binding.MLP(ctx, p)
    X = np.random.default_rng(2).normal(size=(300, 24)).astype(np.float32)
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    want = omlp.forward(p, X)[3]
    # same BF16-rounded operands; FP32 vs FP64 accumulation order only
    assert np.allclose(Y, want, rtol=2e-2, atol=2e-2 * np.abs(want).max())


def _gradient_magnitudes(p, X, T, M):
    """The gradient of the oracle with every term taken by absolute value
    (|h2|^T |dy|, ..., the ReLU masks kept): the sum of the magnitudes of the
    terms that each gradient entry adds up.  Two evaluations of the same
    network on the same BF16 operands differ, entry by entry, by a small
    multiple of the BF16 rounding step times this sum: the FP32 and FP64
    accumulation orders differ, and a hidden activation whose FP32 and FP64
    sums straddle a BF16 rounding boundary rounds to the neighbouring BF16
    value (2^-7 relative) in one of them."""
    W = omlp.unpack(omlp.bf16(p))
    x, h1, h2, y = omlp.forward(p, X)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(1.0, float((M != 0).sum()))
    dy = np.abs(2.0 * M * (y - T) / cnt) + 2.0 * M / cnt * (np.abs(h2) @ np.abs(W["W3"]) + np.abs(W["b3"])) * 2.0 ** -7
    g = {"W3": np.abs(h2).T @ dy, "b3": dy.sum(0)}
    dh2 = (dy @ np.abs(W["W3"]).T) * (h2 > 0)
    g["W2"] = np.abs(h1).T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ np.abs(W["W2"]).T) * (h1 > 0)
    g["W1"] = np.abs(x).T @ dh1
    g["b1"] = dh1.sum(0)
    return g


def test_mlp_backward_matches_oracle(ctx):
    """Every gradient entry of the BF16/FP32 kernels within 2^-6 (two BF16
    rounding steps) of the magnitude sum of its terms from the float64 oracle
    on the same BF16 operands: a BF16 activation that rounds to its neighbour
    moves each term it enters by at most 2^-7 of that term, and the FP32
    accumulation error of these 257-row sums is below 2^-15 of the magnitude
    sum.  Each tensor also within 1e-2 in relative L2 norm; the loss within
    2e-2."""
    import torch
    p = _params(3)
    net = binding.MLP(ctx, p)
    g = np.random.default_rng(4)
    X = g.normal(size=(257, 24)).astype(np.float32)
    T = g.normal(size=(257, 3)).astype(np.float32)
    M = (g.random((257, 3)) < 0.7).astype(np.float32)
    grads, loss = net.backward(*(torch.from_numpy(a).cuda() for a in (X, T, M)))
    lw, gw = omlp.loss_and_grad(p, X, T, M)
    assert float(loss.item()) == pytest.approx(lw, rel=2e-2)
    mag = _gradient_magnitudes(p, X, T, M)
    gg = grads.cpu().numpy().astype(np.float64)
    o = 0
    worst = {}
    for name, shape in omlp.SIZES:
        k = int(np.prod(shape))
        a, b = gg[o:o + k], gw[o:o + k]
        bound = 2.0 ** -6 * mag[name].ravel() + 1e-9
        err = np.abs(a - b)
        worst[name] = float((err / bound).max())
        assert np.all(err <= bound), (name, int(np.argmax(err / bound)), float(err.max()))
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-9, name
        o += k
    print("largest error / bound per tensor:", worst)


def test_mlp_training_fits_a_function(ctx):
    import torch
    g = np.random.default_rng(5)
    X = g.normal(size=(2048, 24)).astype(np.float32)
    A = g.normal(size=(24, 3)).astype(np.float32)
    T = np.tanh(X @ A).astype(np.float32)
    M = np.ones_like(T)
    net = binding.MLP(ctx, omlp.init_params(6))
    Xt, Tt, Mt = (torch.from_numpy(a).cuda() for a in (X, T, M))
    first = None
    for step in range(400):
        idx = torch.from_numpy(g.choice(2048, 256, replace=False)).cuda()
        _, loss = net.backward(Xt[idx], Tt[idx], Mt[idx])
        if first is None:
            first = float(loss.item())
        net.adam(3e-3)
    _, loss = net.backward(Xt, Tt, Mt)
    assert float(loss.item()) < 0.1 * first


def test_features_against_exact_values(ctx):
    R, S, T = datagen.linear_uniform(n=1 << 16, ad=1 << 14, bd=1 << 12, cd=1 << 12, dd=1 << 14, seed=7)
    f = planner.features(ctx, binding.MWJ_LINEAR, cu(R), cu(S), cu(T))
    assert f[0] == pytest.approx(np.log2(1 + 2 ** 16), abs=1e-4)
    for k, col in [(3, R[0]), (4, R[1]), (5, S[1]), (6, T[1])]:
        d = len(np.unique(col))
        assert 2 ** f[k] - 1 == pytest.approx(d, rel=0.06)        # HyperLogLog, 4096 registers
    inter = oracle.binary_count(R, S)
    assert 2 ** f[8] - 1 == pytest.approx(inter, rel=0.05)         # sampled |R join S|
    assert f[7] == 0.0
    # uniform keys: hardly any sampled value repeats 8+ times
    assert f[11] < 0.05


def test_cost_model_orders_plans_by_intermediate_size(ctx):
    small = np.zeros(24, np.float32)
    small[:3] = np.log2(1 + 1e6)
    small[8] = np.log2(1 + 1e5)          # |R join S| far below the inputs
    big = small.copy()
    big[8] = np.log2(1 + 1e10)           # far above
    cs, cb = binding.cost_model(small), binding.cost_model(big)
    assert cb[0] > cs[0] + 5               # the cascade pays for its intermediate
    assert cb[0] > cb[1]                   # and loses to the 3-way join when it is large


def test_trained_network_gains_over_cost_model(ctx):
    """The packaged network (trained on engine timings of instances up to 2^24
    tuples per relation) against the planner without it -- the cost model
    alone -- on held-out instances the engine times now (a seed the training
    never saw, up to 2^20 tuples per relation): a strictly smaller mean regret
    against the best measured plan, and at least as many plans within 10 % of
    it.  Every plan of every instance gave the same total (checked while
    timing); the small instances' totals are checked against the oracle."""
    pl = planner.default_planner(ctx)
    F, times, totals, meta, _ = planner.collect(ctx, 160, 424242, 240.0, size_hi=1 << 20, keep_small=30000)
    assert len(F) >= 100
    summary, _ = planner.evaluate(pl, F, times, [m["sizes"] for m in meta])
    learned, model = summary["learned"], summary["cost_model"]
    print("held-out regret: learned", learned, "cost model", model, "default plan", summary["default"],
          "cascade", summary["cascade"])
    assert learned["mean_regret"] < model["mean_regret"]
    assert learned["within_10pct"] >= model["within_10pct"]
    checked = 0
    for m, tot in zip(meta, totals):
        if "rel" in m:
            fn = oracle.linear if m["kind"] == binding.MWJ_LINEAR else oracle.cyclic
            assert tot == fn(*m["rel"])["total"]
            checked += 1
    assert checked >= 5


def test_trained_planner_plans_are_exact(ctx):
    """The committed network plans real joins; every plan gives the oracle's answer."""
    pl = planner.default_planner(ctx)
    g = np.random.default_rng(21)
    for kind in ["linear", "cyclic", "linear", "cyclic"]:
        q = datagen.random_query(g, kind, size_lo=500, size_hi=20000, dom_lo=50, dom_hi=5000)
        k = binding.MWJ_LINEAR if kind == "linear" else binding.MWJ_CYCLIC
        fn = oracle.linear if kind == "linear" else oracle.cyclic
        want = fn(q.R, q.S, q.T)["total"]
        res, choice = planner.plan_and_run(ctx, k, cu(q.R), cu(q.S), cu(q.T), planner=pl)
        assert int(res["total"].item()) == want, choice
        res, _ = planner.plan_and_run(ctx, k, cu(q.R), cu(q.S), cu(q.T), planner=None)
        assert int(res["total"].item()) == want
        for p in range(3):   # every plan the planner may choose
            assert int(planner.run_plan(ctx, k, cu(q.R), cu(q.S), cu(q.T), p)["total"].item()) == want
