"""Parity of the linear join's aggregates under a skewed join column: heavy
B keys are split off into their own bucket and aggregated by every CTA; the
results must equal the oracle's exactly, whatever the skew and the shares."""
import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import binding, datagen

from factorised import factorised_group_by
from gpu_util import cu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.set_device(0)
    c = binding.Context(0)
    yield c
    c.close()


def check(ctx, R, S, T, a_domain, shares=None):
    dR, dS, dT = cu(R), cu(S), cu(T)
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=a_domain)
    got = ctx.join3_linear(dR, dS, dT, "count", shares=shares)
    assert int(got["total"].item()) == want["total"]
    got = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=shares, a_domain=a_domain)
    assert int(got["total"].item()) == want["total"]
    assert np.array_equal(got["counts"].cpu().numpy(), want["counts"])


@pytest.mark.parametrize("s", [0.8, 1.1, 1.5, 2.0])
@pytest.mark.parametrize("shares", [None, (64, 1), (16, 4), (1, 1), (1024, 1)])
def test_zipf_join_column(ctx, s, shares):
    R, S, T = datagen.skewed_linear(n=1 << 15, s=s, b_domain=1 << 12, c_domain=1 << 10,
                                    a_domain=1 << 10, seed=int(10 * s))
    check(ctx, R, S, T, 1 << 10, shares)


def test_heavy_keys_only_in_one_relation(ctx):
    """Keys heavy in S but absent from R, and heavy in R but light in S."""
    g = np.random.default_rng(3)
    n = 20000
    R = (g.integers(0, 100, n).astype(np.int32),
         np.where(g.random(n) < 0.5, 7, g.integers(100, 5000, n)).astype(np.int32))
    S = (np.where(g.random(n) < 0.5, 9, g.integers(100, 5000, n)).astype(np.int32),
         g.integers(0, 300, n).astype(np.int32))
    T = (g.integers(0, 300, n).astype(np.int32), g.integers(0, 100, n).astype(np.int32))
    check(ctx, R, S, T, 100)
    check(ctx, R, S, T, 100, (64, 1))
    check(ctx, R, S, T, 100, (8, 2))


def test_many_heavy_keys(ctx):
    """More heavy candidates than the heavy table holds: the rest stay light."""
    g = np.random.default_rng(4)
    n = 1 << 16
    b = g.integers(0, 600, n).astype(np.int32)   # 600 keys of ~1/600 share each
    R = (g.integers(0, 64, n).astype(np.int32), b)
    S = (g.permutation(b), g.integers(0, 500, n).astype(np.int32))
    T = (g.integers(0, 500, n).astype(np.int32), g.integers(0, 64, n).astype(np.int32))
    check(ctx, R, S, T, 64, (1024, 1))


def test_skewed_full_size(ctx):
    """The skew workload of the benchmark line: 2^22 tuples per relation,
    B Zipf(1.5) (the top key holds ~38% of R and of S), with the default plan
    (one bucket per side) and the partitioned plan with its heavy-key bucket."""
    R, S, T = datagen.skewed_linear()
    total, cnt = factorised_group_by(R, S, T, 1 << 20)
    dR, dS, dT = cu(R), cu(S), cu(T)
    part = ctx.plan_shares(binding.MWJ_LINEAR, dR, dS, dT, binding.MWJ_MATERIALIZE)
    for shares in (None, part):
        got = ctx.join3_linear(dR, dS, dT, "group_by_a", shares=shares, a_domain=1 << 20)
        assert int(got["total"].item()) == total
        assert np.array_equal(got["counts"].cpu().numpy(), cnt)
        got = ctx.join3_linear(dR, dS, dT, "count", shares=shares)
        assert int(got["total"].item()) == total
