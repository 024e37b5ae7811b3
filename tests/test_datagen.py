"""The seeded input generators follow the recipe the design notes state (the
shapes of the paper's workloads): power-law friend graphs, uniform keys, a
Zipf join column, star schemas.  CPU only; no join arithmetic here beyond
numpy degree sums that pin the workload's sizes."""
import numpy as np
import pytest

from paper_1905_13376_gb300 import datagen


def test_zipf_rank_weights_mean_and_cap():
    w = datagen.zipf_rank_weights(1 << 16, 32.0, s=1.1, cap=4096.0)
    assert w.mean() == pytest.approx(32.0, rel=1e-9)
    assert w.max() == 4096.0 and w[0] == 4096.0          # the top ranks hit the cap
    assert np.all(np.diff(w) <= 0)                      # non-increasing in rank
    r = np.arange(1, len(w) + 1, dtype=np.float64)
    free = w < 4096.0
    c = w[free] * r[free] ** 1.1                        # w_r = c r^-1.1 below the cap
    assert np.allclose(c, c[0], rtol=1e-9)


def test_friends_graph_full_size_recipe():
    """The 2^20-vertex directed Chung-Lu graph of the benchmark: its size,
    its form (sorted by source, no duplicates, no self loops, degrees below
    the cap) and the two join sizes the notes quote."""
    n = 1 << 20
    src, dst = datagen.chung_lu_directed()
    assert src.dtype == np.int32 and dst.dtype == np.int32
    assert len(src) == 32_804_288
    code = src.astype(np.int64) * n + dst
    assert np.all(np.diff(code) > 0)                    # sorted by (src, dst), distinct
    assert not np.any(src == dst)
    assert src.min() >= 0 and dst.min() >= 0 and src.max() < n and dst.max() < n
    outdeg = np.bincount(src, minlength=n).astype(np.int64)
    indeg = np.bincount(dst, minlength=n).astype(np.int64)
    assert outdeg.max() <= 4096 and indeg.max() <= 4096
    assert 30.0 < len(src) / n <= 32.0                  # mean 32 before duplicates are dropped
    # |F |x| F| = sum_v indeg(v) outdeg(v); 3-paths = sum over (a,b) of w(b),
    # w(b) = sum over (b,c) of outdeg(c) (exact in float64: every partial sum < 2^53)
    assert int((indeg * outdeg).sum()) == 1_013_013_234
    w = np.bincount(src, weights=outdeg[dst].astype(np.float64), minlength=n)
    assert int(w[dst].sum()) == 31_268_001_373


def test_generators_are_seeded():
    a = datagen.chung_lu_directed(n_vertices=1 << 12)
    b = datagen.chung_lu_directed(n_vertices=1 << 12)
    c = datagen.chung_lu_directed(n_vertices=1 << 12, seed=datagen.SEED_BASE + 99)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0]) or not np.array_equal(a[1], c[1])
    u = datagen.linear_uniform(n=1000, seed=7)
    v = datagen.linear_uniform(n=1000, seed=7)
    assert all(np.array_equal(x, y) for r, q in zip(u, v) for x, y in zip(r, q))


def test_linear_uniform_domains():
    R, S, T = datagen.linear_uniform(n=1 << 16)
    for col, dom in ((R[0], 1 << 20), (R[1], 1 << 12), (S[0], 1 << 12), (S[1], 1 << 12),
                     (T[0], 1 << 12), (T[1], 1 << 20)):
        assert len(col) == 1 << 16 and col.min() >= 0 and col.max() < dom
    # each key of B appears about n / |B| = 16 times
    assert np.bincount(S[0], minlength=1 << 12).mean() == pytest.approx(16.0)


def test_undirected_graph_orientation():
    a, b = datagen.chung_lu_undirected(n_vertices=1 << 12, mean_degree=16.0)
    assert np.all(a < b)
    code = a.astype(np.int64) * (1 << 12) + b
    assert len(np.unique(code)) == len(code)


def test_skewed_join_column():
    """B Zipf(1.5) over 2^20 keys through one bijection shared by R and S:
    the top key holds about 1 / zeta(1.5) ~ 38% of each, and it is the same
    key in both."""
    n = 1 << 20
    R, S, T = datagen.skewed_linear(n=n)
    hr = np.bincount(R[1], minlength=1 << 20)
    hs = np.bincount(S[0], minlength=1 << 20)
    assert hr.argmax() == hs.argmax()
    h = np.sum(np.arange(1, (1 << 20) + 1, dtype=np.float64) ** -1.5)
    for hist in (hr, hs):
        assert hist.max() / n == pytest.approx(1.0 / h, abs=0.005)
    for col, dom in ((R[0], 1 << 20), (S[1], 1 << 22), (T[0], 1 << 22), (T[1], 1 << 20)):
        assert col.min() >= 0 and col.max() < dom


def test_star_schema_foreign_keys():
    R, S, T = datagen.star_schema(n_fact=1 << 16, n_dim=1 << 10, attr_domain=1 << 8)
    assert np.array_equal(np.sort(R[1]), np.arange(1 << 10))     # unique dimension keys
    assert np.array_equal(np.sort(T[0]), np.arange(1 << 10))
    assert S[0].min() >= 0 and S[0].max() < 1 << 10 and S[1].min() >= 0 and S[1].max() < 1 << 10
    assert np.all(np.diff(S[0]) >= 0)                            # fact sorted by B
    assert R[0].max() < 1 << 8 and T[1].max() < 1 << 8
