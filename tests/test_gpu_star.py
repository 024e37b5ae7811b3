"""Parity of the star 3-way join (CUDA, through the C ABI) with the oracle.

The star join computes the linear query R(A,B) S(B,C) T(C,D), so the
linear oracle is its oracle; the star-schema inputs also have a closed form
(every fact tuple joins one tuple of each dimension)."""
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
    got = ctx.join3_star(dR, dS, dT, "count", shares=shares)
    assert int(got["total"].item()) == want["total"]
    got = ctx.join3_star(dR, dS, dT, "group_by_a", shares=shares, a_domain=a_domain)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])
    if rows:
        n = want["total"]
        wr = oracle.linear(R, S, T, oracle.MATERIALIZE, capacity=n)
        got = ctx.join3_star(dR, dS, dT, "rows", shares=shares, capacity=n + 5)
        assert int(got["n_rows"].item()) == n
        assert int(got["total"].item()) == n
        assert np.array_equal(sorted_rows(got["rows"].cpu().numpy()), wr["rows"])


def star_closed_form(R, S, a_domain):
    ra, rb = R
    inv = np.full(int(rb.max()) + 1, -1, dtype=np.int64)
    inv[rb] = np.arange(len(rb))
    return np.bincount(ra[inv[S[0]]], minlength=a_domain)


def test_star_schema_small(ctx):
    R, S, T = datagen.star_schema(n_fact=1 << 16, n_dim=1 << 12, attr_domain=256,
                                  seed=datagen.SEED_BASE + 60)
    check_all_modes(ctx, R, S, T, 256)


@pytest.mark.parametrize("shares", [None, (1, 1), (3, 5), (64, 1), (1, 200), (0, 7)])
def test_share_invariance(ctx, shares):
    R, S, T = datagen.linear_uniform(n=3000, ad=100, bd=50, cd=40, dd=100, seed=61)
    check_all_modes(ctx, R, S, T, 100, shares=shares)


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_with_duplicates(ctx, seed):
    g = np.random.default_rng(100 + seed)
    nR, nS, nT = (int(g.integers(0, 40)) for _ in range(3))
    dom = int(g.integers(1, 6))
    R = (g.integers(0, 9, nR).astype(np.int32), g.integers(-2, dom, nR).astype(np.int32))
    S = (g.integers(-2, dom, nS).astype(np.int32), g.integers(-2, dom, nS).astype(np.int32))
    T = (g.integers(-2, dom, nT).astype(np.int32), g.integers(0, 9, nT).astype(np.int32))
    check_all_modes(ctx, R, S, T, 9)


def test_extreme_keys(ctx):
    vals = np.array([-2**31, 2**31 - 1, -1, 0, 1, -2], dtype=np.int32)
    g = np.random.default_rng(17)
    n = 900
    R = (g.integers(0, 50, n).astype(np.int32), vals[g.integers(0, 6, n)])
    S = (vals[g.integers(0, 6, n)], vals[g.integers(0, 6, n)])
    T = (vals[g.integers(0, 6, n)], g.integers(-100, 100, n).astype(np.int32))
    check_all_modes(ctx, R, S, T, 50, rows=False)


def test_empty_relations(ctx):
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    R, S, T = datagen.linear_uniform(n=100, ad=10, bd=5, cd=5, dd=10, seed=3)
    for args in [(E, S, T), (R, E, T), (R, S, E), (E, E, E)]:
        check_all_modes(ctx, *args, a_domain=10)


def test_ragged_fact_lengths(ctx):
    """Fact relations whose length is not a multiple of the 16-tuple chunk
    granule or of the CTA count, and misaligned column starts."""
    R, S, T = datagen.star_schema(n_fact=50021, n_dim=777, attr_domain=64,
                                  seed=datagen.SEED_BASE + 62)
    for off in (0, 1, 3):
        S2 = (S[0][off:], S[1][off:])
        check_all_modes(ctx, R, S2, T, 64, rows=(off == 1))


def test_domain_error(ctx):
    R, S, T = datagen.star_schema(n_fact=1000, n_dim=64, attr_domain=16, seed=datagen.SEED_BASE + 63)
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_star(cu(R), cu(S), cu(T), "group_by_a", a_domain=8)
    assert ei.value.status == binding.MWJ_ERR_DOMAIN


def test_capacity_error_reports_exact_count(ctx):
    R, S, T = datagen.star_schema(n_fact=5000, n_dim=128, attr_domain=16, seed=datagen.SEED_BASE + 64)
    with pytest.raises(binding.MwjError) as ei:
        ctx.join3_star(cu(R), cu(S), cu(T), "rows", capacity=100)
    assert ei.value.status == binding.MWJ_ERR_CAPACITY
    assert str(len(S[0])) in str(ei.value)


def test_agrees_with_linear_and_cascade(ctx):
    R, S, T = datagen.star_schema(n_fact=1 << 18, n_dim=1 << 13, attr_domain=1 << 10, zipf=True,
                                  seed=datagen.SEED_BASE + 65)
    dR, dS, dT = cu(R), cu(S), cu(T)
    star = ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=1 << 10)
    lin = ctx.join3_linear(dR, dS, dT, "group_by_a", a_domain=1 << 10)
    cas = ctx.cascade_join(binding.MWJ_LINEAR, dR, dS, dT, "group_by_a", a_domain=1 << 10)
    for r in (lin, cas):
        assert int(r["total"].item()) == int(star["total"].item())
        assert np.array_equal(r["counts"].cpu().numpy(), star["counts"].cpu().numpy())
    assert int(star["total"].item()) == len(S[0])
    assert np.array_equal(star["counts"].cpu().numpy(), star_closed_form(R, S, 1 << 10))


@pytest.mark.parametrize("zipf", [False, True])
def test_star_schema_full_size(ctx, zipf):
    """The star workload at full size (2^26 fact tuples, 2^20-tuple
    dimensions): total and every group count against the closed form."""
    R, S, T = datagen.star_schema(zipf=zipf)
    dR, dS, dT = cu(R), cu(S), cu(T)
    got = ctx.join3_star(dR, dS, dT, "count")
    assert int(got["total"].item()) == len(S[0])
    got = ctx.join3_star(dR, dS, dT, "group_by_a", a_domain=1 << 16)
    assert int(got["total"].item()) == len(S[0])
    assert np.array_equal(got["counts"].cpu().numpy(), star_closed_form(R, S, 1 << 16))
