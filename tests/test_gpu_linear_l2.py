"""Parity of the one-bucket linear plan (shares I = J = 1: S's weight table and
T's table held whole in the L2, nothing partitioned) with the oracle, through
the C ABI.  The aggregates take this plan by default."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_13376_gb300 import binding, datagen

from gpu_util import cu, dev

pytestmark = pytest.mark.gpu

ONE = (1, 1, 1)


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    c = binding.Context(0)
    yield c
    c.close()


def check(ctx, R, S, T, a_domain, rels=None):
    dR, dS, dT = rels if rels is not None else (cu(R), cu(S), cu(T))
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
    got = ctx.join3_linear(dR, dS, dT, "count", shares=ONE)
    assert int(got["total"].item()) == want["total"]
    got = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=ONE, a_domain=a_domain)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
    return want


def test_default_plan_of_aggregates_is_one_bucket(ctx):
    R, S, T = datagen.linear_uniform(n=1000, ad=50, bd=20, cd=20, dd=50, seed=1)
    d = cu(R)
    for mode in (binding.MWJ_COUNT, binding.MWJ_COUNT_GROUP_BY_A):
        assert ctx.plan_shares(binding.MWJ_LINEAR, d, d, d, mode) == ONE
    assert ctx.plan_shares(binding.MWJ_LINEAR, d, d, d, binding.MWJ_MATERIALIZE)[0] > 1


@pytest.mark.parametrize("seed", range(8))
def test_ragged_sizes(ctx, seed):
    """Sizes that end inside a lane's four tuples and inside a warp's 128."""
    g = np.random.default_rng(100 + seed)
    nR, nS, nT = (int(g.integers(1, 700)) for _ in range(3))
    dom = int(g.integers(2, 60))
    R = (g.integers(0, 40, nR).astype(np.int32), g.integers(0, dom, nR).astype(np.int32))
    S = (g.integers(0, dom, nS).astype(np.int32), g.integers(0, dom, nS).astype(np.int32))
    T = (g.integers(0, dom, nT).astype(np.int32), g.integers(0, 9, nT).astype(np.int32))
    check(ctx, R, S, T, 40)


@pytest.mark.parametrize("run", [1, 3, 4, 5, 31, 129, 1000])
def test_sorted_runs_across_lanes_and_warps(ctx, run):
    """Runs of equal keys (edge lists sorted by source) of every length
    relative to a lane's four tuples and a warp's 128: the runs merged inside
    a warp must add up exactly."""
    g = np.random.default_rng(run)
    n = 20000
    keys = np.repeat(np.arange(n // run + 1, dtype=np.int32), run)[:n]
    R = (keys.copy(), g.integers(0, 3000, n).astype(np.int32))          # a sorted, b random
    S = (np.sort(g.integers(0, 3000, n)).astype(np.int32), g.integers(0, 2000, n).astype(np.int32))
    T = (np.sort(g.integers(0, 2000, n)).astype(np.int32), g.integers(0, 5, n).astype(np.int32))
    check(ctx, R, S, T, int(keys.max()) + 1)


def test_unaligned_columns(ctx):
    """Columns that do not start on a 16-byte boundary take the scalar loads."""
    R, S, T = datagen.linear_uniform(n=5001, ad=300, bd=64, cd=64, dd=300, seed=21)

    def off(rel, k):
        return tuple(torch.from_numpy(np.concatenate([np.zeros(k, np.int32), c])).to(dev())[k:]
                     for c in rel)
    for k in (1, 2, 3):
        rels = (off(R, k), off(S, (k + 1) % 4), off(T, k))
        assert any(c.data_ptr() % 16 for rel in rels for c in rel)
        check(ctx, R, S, T, 300, rels=rels)


def test_weights_past_2_pow_32(ctx):
    """w(b) = sum of deg_T(c) over S reaches 2^32 for b = 7 and b = -1 (the
    key kept outside the table): the carry into the high word is exact."""
    k = (1 << 16) + 5
    S = (np.concatenate([np.full(k, 7, np.int32), np.full(k, -1, np.int32),
                         np.arange(100, dtype=np.int32)]),
         np.concatenate([np.full(2 * k, 3, np.int32), np.full(100, 4, np.int32)]))
    T = (np.concatenate([np.full(1 << 16, 3, np.int32), np.full(9, 4, np.int32)]),
         np.arange((1 << 16) + 9, dtype=np.int32))
    R = (np.array([0, 0, 1, 2, 3, 3, 3, 4], np.int32), np.array([7, 7, -1, 5, 7, -1, 6, 99], np.int32))
    want = check(ctx, R, S, T, 5)
    assert int(want["counts"][0]) == 2 * (k * (1 << 16) + 9) > (1 << 33)


@pytest.mark.parametrize("t_spread", [False, True])
@pytest.mark.parametrize("w_spread", [False, True])
def test_table_layouts(ctx, t_spread, w_spread):
    """Both layouts of T's table and of S's weight table, in every pairing:
    the sizing pass gives keys whose range is at most the hashed table's slot
    count the direct-address layout (entry at key - min), and keys spread
    wider the hashed one.  One far-away key that joins nothing (a T tuple
    with C = -2^31, an S tuple with B = 2^30 + 1) spreads a column without
    changing the result.  Weights reach 2^32 (the hashed layout's carry word
    and its key -1 slot, the direct layout's plain 64-bit words)."""
    k = (1 << 16) + 5
    g = np.random.default_rng(41)
    Sb = np.concatenate([np.full(k, 7, np.int32), np.full(k, -1, np.int32),
                         g.integers(-3, 2000, 30000).astype(np.int32)])
    Sc = np.concatenate([np.full(2 * k, 3, np.int32), g.integers(0, 3000, 30000).astype(np.int32)])
    Tc = np.concatenate([np.full(1 << 16, 3, np.int32), g.integers(0, 3000, 20000).astype(np.int32)])
    Td = g.integers(0, 9, len(Tc)).astype(np.int32)
    if w_spread:
        Sb = np.append(Sb, np.int32((1 << 30) + 1))
        Sc = np.append(Sc, np.int32(-5))            # no T tuple has C = -5
    if t_spread:
        Tc = np.append(Tc, np.int32(-2 ** 31))      # no S tuple has C = -2^31
        Td = np.append(Td, np.int32(0))
    Ra = g.integers(0, 50, 40000).astype(np.int32)
    Rb = np.concatenate([np.array([7, 7, -1, 5, 7, -1], np.int32),
                         g.integers(-3, 2100, 40000 - 6).astype(np.int32)])
    want = check(ctx, (Ra, Rb), (Sb, Sc), (Tc, Td), 50)
    assert int(want["total"]) > (1 << 33)


@pytest.mark.parametrize("n", [1023, 1024, 1025, 5000, 3 * 1024 * 152 + 13])
def test_round_boundaries(ctx, n):
    """Sizes around one CTA's 1024 tuples of warp rounds and a run of rounds
    over every SM with a ragged tail, sorted by A and by B so that runs of
    equal keys cross lanes, warps and CTAs."""
    g = np.random.default_rng(n)
    R = (np.sort(g.integers(0, 700, n)).astype(np.int32), g.integers(0, 900, n).astype(np.int32))
    S = (np.sort(g.integers(0, 900, n)).astype(np.int32), g.integers(0, 800, n).astype(np.int32))
    T = (g.integers(0, 800, n).astype(np.int32), g.integers(0, 5, n).astype(np.int32))
    check(ctx, R, S, T, 700)


def test_domain_error(ctx):
    R = (np.array([0, 5, 1], np.int32), np.array([1, 1, 2], np.int32))
    S = (np.array([1, 2], np.int32), np.array([2, 2], np.int32))
    T = (np.array([2], np.int32), np.array([0], np.int32))
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_linear(cu(R), cu(S), cu(T), "group_by_a", shares=ONE, a_domain=5)
    assert ei.value.status == binding.MWJ_ERR_DOMAIN
    # an a outside the domain whose tuple joins nothing is an error all the same
    R = (np.array([0, 9], np.int32), np.array([1, 3], np.int32))
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_linear(cu(R), cu(S), cu(T), "group_by_a", shares=ONE, a_domain=5)
    assert ei.value.status == binding.MWJ_ERR_DOMAIN


def test_many_distinct_keys(ctx):
    """Distinct B and C values in the millions: tables of 2^23+ slots."""
    g = np.random.default_rng(9)
    n = 1 << 21
    R = (g.integers(0, 1 << 16, n).astype(np.int32), g.integers(0, 1 << 30, n).astype(np.int32))
    S = (np.concatenate([R[1][: n // 2], g.integers(0, 1 << 30, n // 2)]).astype(np.int32),
         g.integers(0, 1 << 22, n).astype(np.int32))
    T = (g.integers(0, 1 << 22, n).astype(np.int32), g.integers(0, 100, n).astype(np.int32))
    check(ctx, R, S, T, 1 << 16)


def test_matches_partitioned_plan_on_friends_graph(ctx):
    """The power-law friends graph at 2^18 vertices: the one-bucket plan, the
    partitioned plan and the oracle agree on every group."""
    F = datagen.chung_lu_directed(n_vertices=1 << 18)
    dF = cu(F)
    want = check(ctx, F, F, F, 1 << 18, rels=(dF, dF, dF))
    part = ctx.plan_shares(binding.MWJ_LINEAR, dF, dF, dF, binding.MWJ_MATERIALIZE)
    got = ctx.join3_linear(dF, dF, dF, "group_by_a", shares=part, a_domain=1 << 18)
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
