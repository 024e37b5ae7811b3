"""Parity of the 4-relation chain R(A,B) S(B,C) T(C,D) U(D,E) (CUDA, C ABI)
with the oracle: COUNT and COUNT GROUP BY A, exact."""
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


def check(ctx, R, S, T, U, a_domain, shares=None):
    d = [cu(x) for x in (R, S, T, U)]
    want = oracle.linear4(R, S, T, U, oracle.GROUP_BY_A, a_domain=a_domain)
    got = ctx.join4_linear(*d, "count", shares=shares)
    assert int(got["total"].item()) == want["total"]
    got = ctx.join4_linear(*d, "group_by_a", shares=shares, a_domain=a_domain)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])


def rel(g, n, xd, yd, lo=0):
    return (g.integers(lo, xd, n).astype(np.int32), g.integers(lo, yd, n).astype(np.int32))


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_with_duplicates(ctx, seed):
    g = np.random.default_rng(200 + seed)
    n = [int(g.integers(0, 40)) for _ in range(4)]
    dom = int(g.integers(1, 6))
    R = (g.integers(0, 9, n[0]).astype(np.int32), g.integers(-2, dom, n[0]).astype(np.int32))
    S, T = rel(g, n[1], dom, dom, -2), rel(g, n[2], dom, dom, -2)
    U = (g.integers(-2, dom, n[3]).astype(np.int32), g.integers(0, 9, n[3]).astype(np.int32))
    check(ctx, R, S, T, U, 9)


@pytest.mark.parametrize("shares", [None, (1, 1), (7, 1), (64, 1), (16, 1, 9)])
def test_share_invariance(ctx, shares):
    g = np.random.default_rng(7)
    R, S, T, U = rel(g, 5000, 300, 200), rel(g, 5000, 200, 150), rel(g, 5000, 150, 100), rel(g, 5000, 100, 50)
    check(ctx, R, S, T, U, 300, shares)


def test_many_distinct_keys_chunked(ctx):
    """One H(B) bucket holding ~40K distinct B values: chunked on-chip tables."""
    g = np.random.default_rng(8)
    n = 60000
    R = (g.integers(0, 1000, n).astype(np.int32), g.permutation(n).astype(np.int32))
    S = (g.integers(0, n, n).astype(np.int32), g.integers(0, 3000, n).astype(np.int32))
    T, U = rel(g, n, 3000, 5000), rel(g, n, 5000, 10)
    check(ctx, R, S, T, U, 1000, (1, 1))


def test_extreme_keys(ctx):
    vals = np.array([-2**31, 2**31 - 1, -1, 0, 1, -2], dtype=np.int32)
    g = np.random.default_rng(9)
    n = 700
    R = (g.integers(0, 50, n).astype(np.int32), vals[g.integers(0, 6, n)])
    S = (vals[g.integers(0, 6, n)], vals[g.integers(0, 6, n)])
    T = (vals[g.integers(0, 6, n)], vals[g.integers(0, 6, n)])
    U = (vals[g.integers(0, 6, n)], g.integers(0, 9, n).astype(np.int32))
    check(ctx, R, S, T, U, 50)


def test_one_key_everywhere_and_empty(ctx):
    nR, nS, nT, nU = 300, 40, 500, 700
    R = (np.arange(nR, dtype=np.int32) % 97, np.full(nR, 42, np.int32))
    S = (np.full(nS, 42, np.int32), np.full(nS, -1, np.int32))
    T = (np.full(nT, -1, np.int32), np.full(nT, 5, np.int32))
    U = (np.full(nU, 5, np.int32), np.arange(nU, dtype=np.int32))
    got = ctx.join4_linear(cu(R), cu(S), cu(T), cu(U), "count")
    assert int(got["total"].item()) == nR * nS * nT * nU
    check(ctx, R, S, T, U, 97)
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    for args in [(E, S, T, U), (R, E, T, U), (R, S, E, U), (R, S, T, E)]:
        check(ctx, *args, 97)


def test_rows_mode_rejected(ctx):
    g = np.random.default_rng(10)
    R = rel(g, 10, 5, 5)
    with pytest.raises(binding.MwjError) as ei:
        ctx.join4_linear(cu(R), cu(R), cu(R), cu(R), "rows")
    assert ei.value.status == binding.MWJ_ERR_INVALID_ARG


def test_friends_chain_full_size(ctx):
    """F |x| F |x| F |x| F GROUP BY A on the 2^20-vertex power-law graph."""
    F = datagen.chung_lu_directed()
    check(ctx, F, F, F, F, 1 << 20)
