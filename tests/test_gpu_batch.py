"""Batches of independent joins in one persistent launch (CUDA, through the
C ABI): every query's COUNT equals the oracle, also when the launch is
captured into a CUDA graph and replayed."""
import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import binding, datagen

from gpu_util import cu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.set_device(0)
    c = binding.Context(0)
    yield c
    c.close()


def oracle_count(q):
    fn = oracle.linear if q.kind == "linear" else oracle.cyclic
    return fn(q.R, q.S, q.T)["total"]


def to_batch(ctx, qs, shares=None):
    dev = [(binding.MWJ_LINEAR if q.kind == "linear" else binding.MWJ_CYCLIC,
            cu(q.R), cu(q.S), cu(q.T), None if shares is None else shares[i])
           for i, q in enumerate(qs)]
    return binding.Batch(ctx, dev)


def small_queries(n, seed):
    g = np.random.default_rng(seed)
    return [datagen.random_query(g, "linear" if i % 2 == 0 else "cyclic", size_lo=16,
                                 size_hi=1 << 13, dom_lo=4, dom_hi=1 << 12) for i in range(n)]


def test_batch_matches_oracle(ctx):
    qs = small_queries(300, 1)
    b = to_batch(ctx, qs)
    got = b.launch().cpu().numpy()
    want = np.array([oracle_count(q) for q in qs], dtype=np.int64)
    assert np.array_equal(got, want)
    got2 = b.launch().cpu().numpy()   # a second launch reuses the bound workspace
    assert np.array_equal(got2, want)


def test_batch_with_given_shares_and_empty_queries(ctx):
    g = np.random.default_rng(2)
    qs = [datagen.random_query(g, k, size_lo=50, size_hi=3000, dom_lo=8, dom_hi=300)
          for k in ["linear", "cyclic"] * 10]
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    qs.append(datagen.Query("linear", E, qs[0].S, qs[0].T, qs[0].domains, False))
    qs.append(datagen.Query("cyclic", qs[1].R, E, qs[1].T, qs[1].domains, False))
    shares = [(3, 1, 1) if q.kind == "linear" else (2, 3, 5) for q in qs]
    b = to_batch(ctx, qs, shares)
    got = b.launch().cpu().numpy()
    assert np.array_equal(got, np.array([oracle_count(q) for q in qs], dtype=np.int64))
    assert b.shares(0) == (3, 1, 1)


def test_batch_graph_capture_replay(ctx):
    import torch
    qs = small_queries(120, 3)
    want = np.array([oracle_count(q) for q in qs], dtype=np.int64)
    b = to_batch(ctx, qs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.launch(stream=s)            # first launch binds the workspace, outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.launch(stream=s)
    for _ in range(3):
        b.counts.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(b.counts[: len(qs)].cpu().numpy(), want)


def test_batched_workload_full_size_sampled(ctx):
    """The 4096-query workload (sizes 2^8..2^18, domains 2^6..2^20, uniform or
    Zipf(1.0) keys, linear and cyclic alternating) in one batch; 48 queries,
    the largest ones among them, checked exactly against the oracle."""
    qs = datagen.batched_queries(4096)
    b = to_batch(ctx, qs)
    got = b.launch().cpu().numpy()
    sizes = np.array([len(q.R[0]) + len(q.S[0]) + len(q.T[0]) for q in qs])
    g = np.random.default_rng(4)
    pick = np.unique(np.concatenate([np.argsort(-sizes)[:8], g.choice(len(qs), 40, replace=False)]))
    for i in pick:
        assert got[i] == oracle_count(qs[i]), i


def test_autotuned_batch_is_exact(ctx):
    """Rules tuned on the engine change the plans, never a count: every query
    of a batch created after tuning gives the oracle's count, and restoring
    the library's rules gives the same counts again."""
    from paper_1905_13376_gb300 import autotune
    qs = small_queries(200, 7)
    dev = [(binding.MWJ_LINEAR if q.kind == "linear" else binding.MWJ_CYCLIC, cu(q.R), cu(q.S), cu(q.T))
           for q in qs]
    tuning = autotune.autotune(ctx, dev, context=64, reps=2)
    assert len(tuning["launch"]) == 2 and tuning["context_queries"] == 64
    wb = tuning["whole_batch_ms"]
    # kept only when it beats the library's rule on the whole batch
    if wb["kept"]:
        assert wb["tuned"] < wb["library_rule"]
    else:
        assert tuning["rules"] == [] and tuning["launch"] == [0, 0]
    want = np.array([oracle_count(q) for q in qs], dtype=np.int64)
    b = binding.Batch(ctx, dev)
    assert np.array_equal(b.launch().cpu().numpy(), want)
    # a rule far from the library's: a few R tuples per bucket, every cyclic tile small
    ctx.batch_set_rules([(binding.MWJ_LINEAR, c, 64, 8, 0) for c in range(32)] +
                        [(binding.MWJ_CYCLIC, c, 0, 0, 10) for c in range(32)])
    ctx.batch_set_launch(1, 1)
    b2 = binding.Batch(ctx, dev)
    assert np.array_equal(b2.launch().cpu().numpy(), want)
    assert any(b2.shares(i) != b.shares(i) for i in range(len(qs)))
    ctx.batch_set_rules([])
    ctx.batch_set_launch(0, 0)
    b3 = binding.Batch(ctx, dev)
    assert np.array_equal(b3.launch().cpu().numpy(), want)
