"""Pins of the Flajolet-Martin oracle (Section 4.1's footnote: distinct
friends of friends of friends per person, PCSA sketches)."""
import itertools

import numpy as np
import pytest

from oracle import fm


def test_fof3_sets_brute_force():
    g = np.random.default_rng(1)
    for _ in range(20):
        n = [int(g.integers(0, 12)) for _ in range(3)]
        R = (g.integers(0, 4, n[0]), g.integers(0, 5, n[0]))
        S = (g.integers(0, 5, n[1]), g.integers(0, 5, n[1]))
        T = (g.integers(0, 5, n[2]), g.integers(0, 9, n[2]))
        want = {a: set() for a in range(4)}
        for (a, b), (b2, c), (c2, d) in itertools.product(zip(*R), zip(*S), zip(*T)):
            if b == b2 and c == c2:
                want[int(a)].add(int(d))
        assert fm.fof3_sets(R, S, T, range(4)) == want


def test_hash_avalanche_and_bijection():
    """fmix32 spreads every input bit over all output bits (each output bit
    flips for about half of the inputs) and is one-to-one on a sample."""
    g = np.random.default_rng(2)
    xs = g.integers(0, 2**32, 4000, dtype=np.uint64).tolist()
    hs = [fm.fmix32(x) for x in xs]
    assert len(set(hs)) == len(set(xs))
    for bit in (0, 7, 16, 31):
        flips = np.array([fm.fmix32(x ^ (1 << bit)) ^ h for x, h in zip(xs, hs)], dtype=np.uint64)
        frac = np.array([[(int(f) >> o) & 1 for o in range(32)] for f in flips]).mean(axis=0)
        assert np.all(frac > 0.4) and np.all(frac < 0.6)


def test_bit_distribution():
    """Bitmap index uniform over M; bit k taken with probability 2^-(k+1)."""
    vals = np.arange(200000)
    js = np.zeros(fm.M)
    ks = np.zeros(32)
    for v in vals:
        j, k = fm.bit_of(int(v))
        js[j] += 1
        ks[k] += 1
    assert np.all(np.abs(js / len(vals) - 1 / fm.M) < 0.005)
    for k in range(6):
        assert abs(ks[k] / len(vals) - 2.0 ** -(k + 1)) < 0.01


@pytest.mark.parametrize("n,trials", [(3000, 160), (20000, 64)])
def test_estimator_mean_and_spread(n, trials):
    """PCSA's estimate is unbiased to within a few percent for n >> M and has
    relative standard error ~0.78/sqrt(M) = 0.195 (Flajolet-Martin 1985).
    Bounds sit >= 4 standard errors of the sample mean from 1 (a wrong
    correction factor or bit rule moves the mean by far more)."""
    g = np.random.default_rng(n)
    ratios = []
    for _ in range(trials):
        vals = g.choice(2**31, size=n, replace=False)
        ratios.append(fm.estimate(fm.sketch_of(vals)) / n)
    ratios = np.array(ratios)
    se = 0.21 / np.sqrt(trials)
    assert abs(ratios.mean() - 1.0) < 0.03 + 4 * se
    assert 0.13 < ratios.std() < 0.27


def test_union_is_or_and_duplicates_ignored():
    g = np.random.default_rng(3)
    A = g.integers(0, 10**6, 500)
    B = g.integers(0, 10**6, 700)
    assert np.array_equal(fm.sketch_of(np.concatenate([A, B])), fm.sketch_of(A) | fm.sketch_of(B))
    assert np.array_equal(fm.sketch_of(np.concatenate([A, A])), fm.sketch_of(A))
    assert fm.estimate(np.zeros(fm.M, np.uint32)) == pytest.approx(fm.M / fm.PHI)


def test_csr_sets_match_plain_sets():
    g = np.random.default_rng(4)
    for _ in range(40):
        n = [int(g.integers(0, 60)) for _ in range(3)]
        R = (g.integers(-3, 6, n[0]), g.integers(-3, 9, n[0]))
        S = (g.integers(-3, 9, n[1]), g.integers(-3, 9, n[1]))
        T = (g.integers(-3, 9, n[2]), g.integers(0, 20, n[2]))
        plain = fm.fof3_sets(R, S, T, range(-3, 6))
        csr = fm.fof3_sets_csr(R, S, T, range(-3, 6))
        assert all(set(csr[a].tolist()) == plain[a] for a in plain)
