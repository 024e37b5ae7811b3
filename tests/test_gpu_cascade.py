"""The cascade of binary hash joins (CUDA, through the C ABI) equals the
oracle and the 3-way join, with and without chunking of its intermediate."""
import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import binding, datagen

from gpu_util import cu, sorted_rows

pytestmark = pytest.mark.gpu

LIN, CYC = binding.MWJ_LINEAR, binding.MWJ_CYCLIC
PER_ROW = {(LIN, False): 12, (LIN, True): 12, (CYC, False): 20, (CYC, True): 24}


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.set_device(0)
    c = binding.Context(0)
    yield c
    c.close()


def ws_for_room(ctx, kind, R, S, T, mode, room):
    full = ctx.workspace_size(2 + kind, R, S, T, None, binding.MODES[mode])
    return full - ((1 << 24) - room) * PER_ROW[(kind, mode == "rows")]


def check(ctx, kind, R, S, T, a_domain, room=None, rows=True):
    fn = oracle.linear if kind == LIN else oracle.cyclic
    dR, dS, dT = cu(R), cu(S), cu(T)
    want = fn(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
    modes = ["count", "group_by_a"] + (["rows"] if rows else [])
    for mode in modes:
        wsb = ws_for_room(ctx, kind, dR, dS, dT, mode, room) if room else None
        if mode == "rows":
            n = want["total"]
            got = ctx.cascade_join(kind, dR, dS, dT, "rows", capacity=n + 2, workspace_bytes=wsb)
            wr = fn(R, S, T, oracle.MATERIALIZE, capacity=n)
            assert int(got["n_rows"].item()) == n
            assert np.array_equal(sorted_rows(got["rows"].cpu().numpy()), wr["rows"])
        else:
            got = ctx.cascade_join(kind, dR, dS, dT, mode, a_domain=a_domain, workspace_bytes=wsb)
            assert int(got["total"].item()) == want["total"]
            if mode == "group_by_a":
                assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])


def test_linear_uniform(ctx):
    R, S, T = datagen.linear_uniform(n=2500, ad=400, bd=64, cd=64, dd=400, seed=21)
    check(ctx, LIN, R, S, T, 400)


def test_linear_chunked_intermediate(ctx):
    # |I| = |R join S| ~ 1.6e6 rows through a room of 5e4 rows: ~32 chunks
    R, S, T = datagen.linear_uniform(n=8000, ad=300, bd=40, cd=40, dd=300, seed=22)
    assert oracle.binary_count(R, S) > 20 * 50000
    check(ctx, LIN, R, S, T, 300, room=50000, rows=False)
    g = np.random.default_rng(25)
    R = (g.integers(0, 100, 1500).astype(np.int32), g.integers(0, 10, 1500).astype(np.int32))
    S = (g.integers(0, 10, 1500).astype(np.int32), g.integers(0, 40, 1500).astype(np.int32))
    T = (g.integers(0, 40, 500).astype(np.int32), g.integers(0, 100, 500).astype(np.int32))
    check(ctx, LIN, R, S, T, 100, room=50000)


@pytest.mark.parametrize("seed", range(5))
def test_linear_random_bags(ctx, seed):
    g = np.random.default_rng(300 + seed)
    dom = int(g.integers(1, 6))
    nR, nS, nT = (int(g.integers(0, 40)) for _ in range(3))
    R = (g.integers(0, 7, nR).astype(np.int32), g.integers(-1, dom, nR).astype(np.int32))
    S = (g.integers(-1, dom, nS).astype(np.int32), g.integers(-1, dom, nS).astype(np.int32))
    T = (g.integers(-1, dom, nT).astype(np.int32), g.integers(0, 7, nT).astype(np.int32))
    check(ctx, LIN, R, S, T, 7)


def test_linear_skewed(ctx):
    g = np.random.default_rng(23)
    q = datagen.random_query(g, "linear", size_lo=5000, size_hi=9000, dom_lo=100, dom_hi=500,
                             zipf=True, zipf_s=1.2)
    check(ctx, LIN, q.R, q.S, q.T, q.domains[0], rows=False)


def test_cyclic_triangles(ctx):
    a, b = datagen.chung_lu_undirected(n_vertices=1 << 13, mean_degree=16.0, seed=31)
    R, S, T = datagen.triangle_relations(a, b)
    check(ctx, CYC, R, S, T, 1 << 13)


def test_cyclic_chunked_intermediate(ctx):
    a, b = datagen.chung_lu_undirected(n_vertices=1 << 13, mean_degree=24.0, seed=32)
    R, S, T = datagen.triangle_relations(a, b)
    check(ctx, CYC, R, S, T, 1 << 13, room=20000)


@pytest.mark.parametrize("seed", range(5))
def test_cyclic_random_bags(ctx, seed):
    g = np.random.default_rng(400 + seed)
    da, db, dc = (int(g.integers(1, 5)) for _ in range(3))
    nR, nS, nT = (int(g.integers(0, 40)) for _ in range(3))
    R = (g.integers(0, da, nR).astype(np.int32), g.integers(-1, db, nR).astype(np.int32))
    S = (g.integers(-1, db, nS).astype(np.int32), g.integers(-1, dc, nS).astype(np.int32))
    T = (g.integers(-1, dc, nT).astype(np.int32), g.integers(0, da, nT).astype(np.int32))
    check(ctx, CYC, R, S, T, max(da, 1))


def test_multiway_equals_cascade_friends(ctx):
    F = datagen.chung_lu_directed(n_vertices=1 << 14, mean_degree=32.0, seed=33)
    dF = cu(F)
    mw = ctx.join3_linear(dF, dF, dF, "group_by_a", a_domain=1 << 14)
    cs = ctx.cascade_join(LIN, dF, dF, dF, "group_by_a", a_domain=1 << 14)
    assert int(mw["total"].item()) == int(cs["total"].item())
    assert np.array_equal(mw["counts"].cpu().numpy(), cs["counts"].cpu().numpy())


def test_cascade_errors(ctx):
    R, S, T = datagen.linear_uniform(n=300, ad=10, bd=6, cd=6, dd=10, seed=24)
    dR, dS, dT = cu(R), cu(S), cu(T)
    n = oracle.linear(R, S, T)["total"]
    with pytest.raises(binding.MwjError) as ei:
        ctx.cascade_join(LIN, dR, dS, dT, "rows", capacity=n - 1)
    assert ei.value.status == binding.MWJ_ERR_CAPACITY
    with pytest.raises(binding.MwjError) as ei:
        ctx.cascade_join(LIN, dR, dS, dT, "group_by_a", a_domain=5)
    assert ei.value.status == binding.MWJ_ERR_DOMAIN
