"""Parity of the linear 3-way join (CUDA, through the C ABI) with the oracle."""
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
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
    got = ctx.join3_linear(dR, dS, dT, "count", shares=shares)
    assert int(got["total"].item()) == want["total"]
    got = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=shares, a_domain=a_domain)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
    if rows:
        n = want["total"]
        wr = oracle.linear(R, S, T, oracle.MATERIALIZE, capacity=n)
        got = ctx.join3_linear(dR, dS, dT, "rows", shares=shares, capacity=n + 5)
        assert int(got["n_rows"].item()) == n
        assert np.array_equal(sorted_rows(got["rows"].cpu().numpy()), wr["rows"])


def test_uniform_small(ctx):
    R, S, T = datagen.linear_uniform(n=2000, ad=300, bd=64, cd=64, dd=300, seed=11)
    check_all_modes(ctx, R, S, T, 300)


@pytest.mark.parametrize("shares", [(1, 1), (3, 1), (7, 5), (64, 1), (16, 16), (1, 200)])
def test_share_invariance(ctx, shares):
    R, S, T = datagen.linear_uniform(n=3000, ad=100, bd=50, cd=40, dd=100, seed=12)
    check_all_modes(ctx, R, S, T, 100, shares=shares)


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_with_duplicates(ctx, seed):
    g = np.random.default_rng(seed)
    nR, nS, nT = (int(g.integers(0, 40)) for _ in range(3))
    dom = int(g.integers(1, 6))
    R = (g.integers(0, 9, nR).astype(np.int32), g.integers(-2, dom, nR).astype(np.int32))
    S = (g.integers(-2, dom, nS).astype(np.int32), g.integers(-2, dom, nS).astype(np.int32))
    T = (g.integers(-2, dom, nT).astype(np.int32), g.integers(0, 9, nT).astype(np.int32))
    check_all_modes(ctx, R, S, T, 9)


def test_extreme_keys(ctx):
    vals = np.array([-2**31, 2**31 - 1, -1, 0, 1, -2], dtype=np.int32)
    g = np.random.default_rng(7)
    n = 900
    R = (g.integers(0, 50, n).astype(np.int32), vals[g.integers(0, 6, n)])
    S = (vals[g.integers(0, 6, n)], vals[g.integers(0, 6, n)])
    T = (vals[g.integers(0, 6, n)], g.integers(-100, 100, n).astype(np.int32))
    check_all_modes(ctx, R, S, T, 50, rows=False)
    check_all_modes(ctx, (R[0][:1], R[1][:1]), S, T, 50)


def test_empty_relations(ctx):
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    R, S, T = datagen.linear_uniform(n=100, ad=10, bd=5, cd=5, dd=10, seed=3)
    for args in [(E, S, T), (R, E, T), (R, S, E), (E, E, E)]:
        check_all_modes(ctx, *args, a_domain=10)


def test_single_key_everywhere(ctx):
    nR, nS, nT = 3000, 50, 2000
    R = (np.arange(nR, dtype=np.int32) % 97, np.full(nR, 42, np.int32))
    S = (np.full(nS, 42, np.int32), np.full(nS, -1, np.int32))
    T = (np.full(nT, -1, np.int32), np.arange(nT, dtype=np.int32))
    check_all_modes(ctx, R, S, T, 97, rows=False)
    got = ctx.join3_linear(cu(R), cu(S), cu(T), "count")
    assert int(got["total"].item()) == nR * nS * nT


def test_many_distinct_keys_in_one_bucket_chunks(ctx):
    # I = 1: all of R's ~60K distinct B values land in one on-chip table,
    # which forces the chunked build; the result must not change
    g = np.random.default_rng(5)
    n = 60000
    R = (g.integers(0, 1000, n).astype(np.int32), g.permutation(n).astype(np.int32))
    S = (g.integers(0, n, n).astype(np.int32), g.integers(0, 3000, n).astype(np.int32))
    T = (g.integers(0, 3000, n).astype(np.int32), g.integers(0, 10, n).astype(np.int32))
    check_all_modes(ctx, R, S, T, 1000, shares=(1, 1))
    check_all_modes(ctx, R, S, T, 1000, shares=(2, 1))
    check_all_modes(ctx, R, S, T, 1000, shares=(2, 3))


@pytest.mark.parametrize("nR,nS", [(20000, 60000), (60000, 20000), (30000, 30000)])
def test_build_side_and_chunks(ctx, nR, nS):
    """|S| > 2|R| keeps R_i on chip (Algorithm 1's roles); otherwise S_i is
    the on-chip side of the aggregates.  With few buckets either side holds
    more distinct B values than one table, so both run in chunks."""
    g = np.random.default_rng(nR + 7 * nS)
    R = (g.integers(0, 500, nR).astype(np.int32), g.integers(0, 40000, nR).astype(np.int32))
    S = (g.integers(0, 40000, nS).astype(np.int32), g.integers(0, 2000, nS).astype(np.int32))
    T = (g.integers(0, 2000, 5000).astype(np.int32), g.integers(0, 10, 5000).astype(np.int32))
    for shares in [(1, 1), (4, 1), (64, 1), (8, 4), (16, 1, 9)]:
        check_all_modes(ctx, R, S, T, 500, shares=shares, rows=False)


def test_skewed_zipf(ctx):
    g = np.random.default_rng(8)
    q = datagen.random_query(g, "linear", size_lo=20000, size_hi=40000, dom_lo=200, dom_hi=2000,
                             zipf=True, zipf_s=1.4)
    check_all_modes(ctx, q.R, q.S, q.T, q.domains[0], rows=False)


def test_domain_error(ctx):
    R = (np.array([0, 5, 1], np.int32), np.array([1, 1, 2], np.int32))
    S = (np.array([1, 2], np.int32), np.array([2, 2], np.int32))
    T = (np.array([2], np.int32), np.array([0], np.int32))
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_linear(cu(R), cu(S), cu(T), "group_by_a", a_domain=5)
    assert ei.value.status == binding.MWJ_ERR_DOMAIN


def test_capacity_error_reports_exact_count(ctx):
    R, S, T = datagen.linear_uniform(n=500, ad=10, bd=8, cd=8, dd=10, seed=4)
    n = oracle.linear(R, S, T)["total"]
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_linear(cu(R), cu(S), cu(T), "rows", capacity=n - 1)
    assert ei.value.status == binding.MWJ_ERR_CAPACITY
    assert str(n) in str(ei.value)


def test_aliased_self_join(ctx):
    # F join F join F with R = S = T the same device arrays
    g = np.random.default_rng(2)
    F = (g.integers(0, 700, 20000).astype(np.int32), g.integers(0, 700, 20000).astype(np.int32))
    dF = cu(F)
    want = oracle.linear(F, F, F, oracle.GROUP_BY_A, a_domain=700)
    got = ctx.join3_linear(dF, dF, dF, "group_by_a", a_domain=700)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])


def partitioned(ctx, R, S, T):
    """The library's partitioned plan (its default for row output)."""
    return ctx.plan_shares(binding.MWJ_LINEAR, R, S, T, binding.MWJ_MATERIALIZE)


def test_uniform_config_full_size(ctx):
    R, S, T = datagen.linear_uniform()
    check_all_modes(ctx, R, S, T, 1 << 20, rows=False)
    dR = cu(R)
    check_all_modes(ctx, R, S, T, 1 << 20, shares=partitioned(ctx, dR, dR, dR), rows=False)


def test_friends_workload_full_size(ctx):
    """F |x| F |x| F GROUP BY A on the 2^20-vertex power-law graph, the benchmark
    workload, with the default plan (one bucket per side) and the partitioned
    plan: every count exact."""
    F = datagen.chung_lu_directed()
    dF = cu(F)
    want = oracle.linear(F, F, F, oracle.GROUP_BY_A, a_domain=1 << 20)
    for shares in (None, partitioned(ctx, dF, dF, dF)):
        got = ctx.join3_linear(dF, dF, dF, "group_by_a", shares=shares, a_domain=1 << 20)
        assert int(got["total"].item()) == want["total"]
        assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
        got = ctx.join3_linear(dF, dF, dF, "count", shares=shares)
        assert int(got["total"].item()) == want["total"]


def test_bounded_wait_gives_up_and_context_stays_usable(ctx):
    """A wait on a barrier phase that nothing completes gives up after its
    poll limit: MWJ_ERR_TIMEOUT reaches the host through the status word,
    which is cleared by reading it, and the next join on the context is exact."""
    R, S, T = datagen.linear_uniform(n=4000, ad=500, bd=64, cd=64, dd=500, seed=32)
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=500)
    for polls in (1, 1000):
        assert ctx.check_bounded_wait(polls) == binding.MWJ_ERR_TIMEOUT
        got = ctx.join3_linear(cu(R), cu(S), cu(T), "group_by_a", a_domain=500)
        assert int(got["total"].item()) == want["total"]
        assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])


def test_bounded_wait_runs_out_then_context_recovers(ctx):
    """A context whose device waits give up after one poll: the partitioned
    plan with R's buckets on chip stages their tiles through bulk copies and
    waits on the copies' barriers, so a call either lands every copy in time (the oracle's result)
    or reports MWJ_ERR_TIMEOUT from the status word, each waiting CTA having
    drained its copies in flight before it returned.  A following call on a
    context with the default limit is exact."""
    # |S| > 2|R| keeps R's buckets on chip (Algorithm 1's roles), whose tiles
    # arrive by bulk copies
    g = np.random.default_rng(31)
    nR, nS, nT = 1 << 14, 3 << 14, 1 << 14
    R = (g.integers(0, 1 << 10, nR).astype(np.int32), g.integers(0, 1 << 9, nR).astype(np.int32))
    S = (g.integers(0, 1 << 9, nS).astype(np.int32), g.integers(0, 1 << 9, nS).astype(np.int32))
    T = (g.integers(0, 1 << 9, nT).astype(np.int32), g.integers(0, 1 << 10, nT).astype(np.int32))
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=1 << 10)
    dR, dS, dT = cu(R), cu(S), cu(T)
    impatient = binding.Context(0, spin_limit=1)
    outcomes = set()
    try:
        for _ in range(3):
            try:
                got = impatient.join3_linear(dR, dS, dT, "group_by_a", shares=(64, 1, 1), a_domain=1 << 10)
                assert int(got["total"].item()) == want["total"]
                assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
                outcomes.add("ok")
            except binding.MwjError as e:
                assert e.status == binding.MWJ_ERR_TIMEOUT, e
                outcomes.add("timeout")
    finally:
        impatient.close()
    print("outcomes with a one-poll wait limit:", sorted(outcomes))
    got = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=(64, 1, 1), a_domain=1 << 10)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
