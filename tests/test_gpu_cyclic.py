"""Parity of the cyclic 3-way (triangle) join, CUDA through the C ABI, with the oracle."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import binding, datagen

from gpu_util import cu, sorted_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.set_device(0)
    c = binding.Context(0)
    yield c
    c.close()


def check_all_modes(ctx, R, S, T, a_domain, shares=None, rows=True):
    dR, dS, dT = cu(R), cu(S), cu(T)
    want = oracle.cyclic(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
    got = ctx.join3_cyclic(dR, dS, dT, "count", shares=shares)
    assert int(got["total"].item()) == want["total"]
    got = ctx.join3_cyclic(dR, dS, dT, "group_by_a", shares=shares, a_domain=a_domain)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
    if rows:
        n = want["total"]
        wr = oracle.cyclic(R, S, T, oracle.MATERIALIZE, capacity=n)
        got = ctx.join3_cyclic(dR, dS, dT, "rows", shares=shares, capacity=n + 3)
        assert int(got["n_rows"].item()) == n
        assert np.array_equal(sorted_rows(got["rows"].cpu().numpy()), wr["rows"])


def oriented(edges):
    a = np.array([min(u, v) for u, v in edges], dtype=np.int32)
    b = np.array([max(u, v) for u, v in edges], dtype=np.int32)
    return datagen.triangle_relations(a, b)


@pytest.mark.parametrize("n", [3, 10, 60])
def test_complete_graph(ctx, n):
    R, S, T = oriented(list(itertools.combinations(range(n), 2)))
    got = ctx.join3_cyclic(cu(R), cu(S), cu(T), "count")
    assert int(got["total"].item()) == math.comb(n, 3)
    check_all_modes(ctx, R, S, T, n)


@pytest.mark.parametrize("shares", [(1, 1, 1), (3, 5, 7), (16, 1, 1), (1, 16, 1), (1, 1, 16),
                                    (8, 8, 8), (1, 1, 7), (1, 1, 4096)])
def test_share_invariance(ctx, shares):
    """Cube tilings (x, y, z) and the C-bucket plan (1, 1, z: R whole, grouped
    by B; S and T split by F(c)) give the oracle's result."""
    a, b = datagen.chung_lu_undirected(n_vertices=1 << 12, mean_degree=12.0, seed=77)
    R, S, T = datagen.triangle_relations(a, b)
    check_all_modes(ctx, R, S, T, 1 << 12, shares=shares)


@pytest.mark.parametrize("seed", range(6))
def test_random_bags(ctx, seed):
    g = np.random.default_rng(200 + seed)
    da, db, dc = (int(g.integers(1, 6)) for _ in range(3))
    nR, nS, nT = (int(g.integers(0, 50)) for _ in range(3))
    R = (g.integers(0, da, nR).astype(np.int32), g.integers(-1, db, nR).astype(np.int32))
    S = (g.integers(-1, db, nS).astype(np.int32), g.integers(-1, dc, nS).astype(np.int32))
    T = (g.integers(-1, dc, nT).astype(np.int32), g.integers(0, da, nT).astype(np.int32))
    check_all_modes(ctx, R, S, T, max(da, 1))


def test_extreme_keys_and_minus_one_pairs(ctx):
    vals = np.array([-2**31, 2**31 - 1, -1, 0, 5], dtype=np.int32)
    g = np.random.default_rng(9)
    n = 400
    R = (g.integers(0, 5, n).astype(np.int32), vals[g.integers(0, 5, n)])
    S = (vals[g.integers(0, 5, n)], vals[g.integers(0, 5, n)])
    T = (vals[g.integers(0, 5, n)], g.integers(0, 5, n).astype(np.int32))
    check_all_modes(ctx, R, S, T, 5, rows=False)
    # T tuples equal to (-1, -1) as a (c, a) pair need a domain containing a = -1:
    R2 = (np.full(7, -1, np.int32), np.array([3, 3, 4, -1, 3, 0, 0], np.int32))
    S2 = (np.array([3, -1, 4, 3], np.int32), np.array([-1, -1, -1, 2], np.int32))
    T2 = (np.array([-1, -1, 2], np.int32), np.array([-1, -1, -1], np.int32))
    want = oracle.cyclic(R2, S2, T2)["total"]
    assert want > 0
    assert int(ctx.join3_cyclic(cu(R2), cu(S2), cu(T2), "count")["total"].item()) == want


def test_empty(ctx):
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    R, S, T = oriented([(0, 1), (1, 2), (0, 2)])
    for args in [(E, S, T), (R, E, T), (R, S, E)]:
        check_all_modes(ctx, *args, a_domain=3)


def test_default_plan_is_c_buckets(ctx):
    a, b = datagen.chung_lu_undirected(n_vertices=1 << 12, mean_degree=12.0, seed=78)
    R, S, T = datagen.triangle_relations(a, b)
    sh = ctx.plan_shares(binding.MWJ_CYCLIC, cu(R), cu(S), cu(T))
    assert sh[0] == 1 and sh[1] == 1 and sh[2] >= 1


def test_c_buckets_hashed_b_keys_and_chunks(ctx):
    """B values spread over int32 (R's grouping takes the hashed layout) and
    one C value carrying more T tuples than a bucket's on-chip chunk (the
    bucket is taken in several chunks, S_k streamed past each)."""
    g = np.random.default_rng(13)
    n = 30000
    bvals = g.integers(-2 ** 31, 2 ** 31 - 1, 500).astype(np.int32)
    R = (g.integers(0, 400, n).astype(np.int32), bvals[g.integers(0, 500, n)])
    S = (bvals[g.integers(0, 500, n)], np.where(g.random(n) < 0.3, 7, g.integers(0, 100, n)).astype(np.int32))
    T = (np.concatenate([np.full(20000, 7, np.int32), g.integers(0, 100, 10000).astype(np.int32)]),
         g.integers(0, 400, 30000).astype(np.int32))
    for shares in [None, (1, 1, 1), (1, 1, 3)]:
        check_all_modes(ctx, R, S, T, 400, shares=shares, rows=False)


@pytest.mark.parametrize("copies", [3, 4095, 4097, 70000])
def test_c_buckets_repeated_pairs(ctx, copies):
    """T holds one (c, a) pair many times (a bag): within one on-chip chunk,
    split across a bucket's chunks, and in a big bucket's L2 set.  Each
    distinct pair takes one slot with its multiplicity; every wedge it
    closes counts (and is written) that many times."""
    g = np.random.default_rng(copies)
    T = (np.concatenate([np.full(copies, 9, np.int32), g.integers(0, 50, 3000).astype(np.int32)]),
         np.concatenate([np.full(copies, 3, np.int32), g.integers(0, 40, 3000).astype(np.int32)]))
    R = (np.concatenate([np.full(5, 3, np.int32), g.integers(0, 40, 2000).astype(np.int32)]),
         np.concatenate([np.arange(5, dtype=np.int32), g.integers(0, 30, 2000).astype(np.int32)]))
    S = (np.concatenate([np.arange(5, dtype=np.int32), g.integers(0, 30, 2000).astype(np.int32)]),
         np.concatenate([np.full(5, 9, np.int32), g.integers(0, 50, 2000).astype(np.int32)]))
    want = oracle.cyclic(R, S, T)["total"]
    assert want >= 5 * copies
    for shares in [None, (1, 1, 1), (1, 1, 4)]:
        check_all_modes(ctx, R, S, T, 40, shares=shares)


def test_c_buckets_small_t_large_s(ctx):
    """A small T (one or a few C buckets) and a large S: each bucket's S_k is
    split into work items of its own (the bucket's set rebuilt for each), so
    that the probe is spread over the GPU; every S chunk boundary, ragged
    tail and shares (1, 1, z) give the oracle's result."""
    g = np.random.default_rng(31)
    nR, nS, nT = 5003, 300007, 517
    R = (g.integers(0, 40, nR).astype(np.int32), g.integers(0, 50, nR).astype(np.int32))
    S = (g.integers(0, 50, nS).astype(np.int32), g.integers(0, 60, nS).astype(np.int32))
    T = (g.integers(0, 60, nT).astype(np.int32), g.integers(0, 40, nT).astype(np.int32))
    for shares in [None, (1, 1, 2), (1, 1, 8)]:
        check_all_modes(ctx, R, S, T, 40, shares=shares, rows=shares is None)


def test_c_buckets_tiny_a_domain_zipf_c(ctx):
    """A large T over a tiny A domain with a Zipf C column: T's busiest C
    values repeat each (c, a) pair thousands of times, in big buckets' L2
    sets and in on-chip chunks alike.  Exact, in the time of its wedges."""
    g = np.random.default_rng(71)
    nR, nS, nT = 16597, 231622, 1 << 21
    R = (g.integers(0, 71, nR).astype(np.int32), datagen._keys(g, nR, 43767, True, 1.07))
    S = (datagen._keys(g, nS, 43767, True, 1.07), datagen._keys(g, nS, 400000, True, 1.07))
    T = (datagen._keys(g, nT, 400000, True, 1.07), g.integers(0, 71, nT).astype(np.int32))
    check_all_modes(ctx, R, S, T, 71, rows=False)


def test_big_tiles_split_into_items(ctx):
    # one tile (shares 1,1,1) with R and T far above a chunk: many work items
    g = np.random.default_rng(4)
    n = 20000
    R = (g.integers(0, 300, n).astype(np.int32), g.integers(0, 200, n).astype(np.int32))
    S = (g.integers(0, 200, n).astype(np.int32), g.integers(0, 100, n).astype(np.int32))
    T = (g.integers(0, 100, n).astype(np.int32), g.integers(0, 300, n).astype(np.int32))
    check_all_modes(ctx, R, S, T, 300, shares=(1, 1, 1), rows=False)
    check_all_modes(ctx, R, S, T, 300, shares=(2, 2, 3), rows=False)


def test_skewed_zipf(ctx):
    g = np.random.default_rng(12)
    q = datagen.random_query(g, "cyclic", size_lo=8000, size_hi=16000, dom_lo=100, dom_hi=1000,
                             zipf=True, zipf_s=1.3)
    check_all_modes(ctx, q.R, q.S, q.T, q.domains[0], rows=False)


def test_domain_and_capacity_errors(ctx):
    R, S, T = oriented([(0, 1), (1, 2), (0, 2), (2, 3), (1, 3)])
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_cyclic(cu(R), cu(S), cu(T), "group_by_a", a_domain=1)
    assert ei.value.status == binding.MWJ_ERR_DOMAIN
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_cyclic(cu(R), cu(S), cu(T), "rows", capacity=1)
    assert ei.value.status == binding.MWJ_ERR_CAPACITY


def test_powerlaw_graph_medium(ctx):
    a, b = datagen.chung_lu_undirected(n_vertices=1 << 16, mean_degree=32.0, seed=5)
    R, S, T = datagen.triangle_relations(a, b)
    check_all_modes(ctx, R, S, T, 1 << 16, rows=True)


def test_triangle_workload_full_size_sampled(ctx):
    """2^22-vertex power-law graph (the triangle workload at full size): GPU
    GROUP BY A checked exactly on a sample of A values (the oracle joined with
    R restricted to them, the busiest A values included), sum(counts) ==
    total == the COUNT mode's total == the materialised row count; the full
    triangle list is materialised (capacity from the count) and its rows with
    a sampled A, sorted, equal the oracle's rows for the restricted R."""
    import torch
    a, b = datagen.chung_lu_undirected()
    R, S, T = datagen.triangle_relations(a, b)
    dR, dS, dT = cu(R), cu(S), cu(T)
    n_v = 1 << 22
    got = ctx.join3_cyclic(dR, dS, dT, "group_by_a", a_domain=n_v)
    total = int(got["total"].item())
    counts = got["counts"].cpu().numpy()
    del got
    assert int(counts.sum()) == total
    g = np.random.default_rng(1)
    hubs = np.argsort(-np.bincount(a))[:5].astype(np.int32)   # the busiest A values too
    sample = np.unique(np.concatenate([g.choice(a, 300), hubs]))
    keep = np.isin(R[0], sample)
    Rs = (R[0][keep], R[1][keep])
    want = oracle.cyclic(Rs, S, T, oracle.GROUP_BY_A, a_domain=n_v)
    assert np.array_equal(counts[sample], want["counts"][sample])
    assert int(ctx.join3_cyclic(dR, dS, dT, "count")["total"].item()) == total
    # the materialised list: exactly `total` rows, and the sampled A values'
    # rows equal the oracle's
    got = ctx.join3_cyclic(dR, dS, dT, "rows", capacity=total)
    assert int(got["n_rows"].item()) == total
    rows = got["rows"][:total]
    assert rows.shape == (total, 3)
    mask = torch.isin(rows[:, 0], torch.from_numpy(sample).to(rows.device))
    mine = rows[mask].cpu().numpy()
    # every row is a triangle a < b < c of the oriented graph (checked on the sample)
    assert np.all(mine[:, 0] < mine[:, 1]) and np.all(mine[:, 1] < mine[:, 2])
    del got, rows, mask
    wr = oracle.cyclic(Rs, S, T, oracle.MATERIALIZE, capacity=int(want["total"]))
    assert np.array_equal(sorted_rows(mine), wr["rows"])
