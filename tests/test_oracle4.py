"""The 4-relation chain oracle R(A,B) S(B,C) T(C,D) U(D,E) (Section 7's
"additional levels of hashing beyond two levels"), pinned by brute force,
closed forms and its reduction to the 3-way join."""
import itertools

import numpy as np
import pytest

import oracle


def brute4(R, S, T, U, a_domain):
    cnt = np.zeros(a_domain, dtype=np.int64)
    tot = 0
    for (a, b), (b2, c), (c2, d), (d2, e) in itertools.product(zip(*R), zip(*S), zip(*T), zip(*U)):
        if b == b2 and c == c2 and d == d2:
            cnt[a] += 1
            tot += 1
    return tot, cnt


def rel(g, n, xd, yd, lo=0):
    return (g.integers(lo, xd, n).astype(np.int32), g.integers(lo, yd, n).astype(np.int32))


@pytest.mark.parametrize("seed", range(8))
def test_linear4_vs_brute_force(oracle_lib, seed):
    g = np.random.default_rng(seed)
    n = [int(g.integers(0, 9)) for _ in range(4)]
    dom = int(g.integers(1, 4))
    R = (g.integers(0, 5, n[0]).astype(np.int32), g.integers(-1, dom, n[0]).astype(np.int32))
    S = rel(g, n[1], dom, dom, -1)
    T = rel(g, n[2], dom, dom, -1)
    U = (g.integers(-1, dom, n[3]).astype(np.int32), g.integers(0, 7, n[3]).astype(np.int32))
    tot, cnt = brute4(R, S, T, U, 5)
    got = oracle.linear4(R, S, T, U, oracle.GROUP_BY_A, a_domain=5)
    assert got["total"] == tot
    assert np.array_equal(got["counts"], cnt)
    assert oracle.linear4(R, S, T, U, oracle.COUNT)["total"] == tot


def test_linear4_one_key_everywhere(oracle_lib):
    nR, nS, nT, nU = 7, 5, 11, 13
    R = (np.arange(nR, dtype=np.int32), np.full(nR, 3, np.int32))
    S = (np.full(nS, 3, np.int32), np.full(nS, -5, np.int32))
    T = (np.full(nT, -5, np.int32), np.full(nT, 2**31 - 1, np.int32))
    U = (np.full(nU, 2**31 - 1, np.int32), np.arange(nU, dtype=np.int32))
    got = oracle.linear4(R, S, T, U, oracle.GROUP_BY_A, a_domain=nR)
    assert got["total"] == nR * nS * nT * nU
    assert np.array_equal(got["counts"], np.full(nR, nS * nT * nU))


def test_linear4_factorised(oracle_lib):
    """cnt(a) = sum_{(a,b)} sum_{(b,c)} sum_{(c,d)} deg_U(d), with numpy."""
    g = np.random.default_rng(11)
    R = rel(g, 3000, 64, 40)
    S = rel(g, 3000, 40, 50)
    T = rel(g, 3000, 50, 60)
    U = rel(g, 3000, 60, 99)
    degU = np.bincount(U[0], minlength=60)
    wT = np.bincount(T[0], weights=degU[T[1]], minlength=50).astype(np.int64)
    wS = np.bincount(S[0], weights=wT[S[1]], minlength=40).astype(np.int64)
    cnt = np.bincount(R[0], weights=wS[R[1]], minlength=64).astype(np.int64)
    got = oracle.linear4(R, S, T, U, oracle.GROUP_BY_A, a_domain=64)
    assert np.array_equal(got["counts"], cnt)
    assert got["total"] == int(cnt.sum())


def test_linear4_reduces_to_linear3(oracle_lib):
    """With U = {(d, 0)} holding each D value once, deg_U(d) = 1 for every d
    in U and the chain counts exactly the 3-way join restricted to those d."""
    g = np.random.default_rng(12)
    R, S, T = rel(g, 2000, 100, 30), rel(g, 2000, 30, 30), rel(g, 2000, 30, 80)
    U = (np.arange(80, dtype=np.int32), np.zeros(80, np.int32))
    want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=100)
    got = oracle.linear4(R, S, T, U, oracle.GROUP_BY_A, a_domain=100)
    assert got["total"] == want["total"]
    assert np.array_equal(got["counts"], want["counts"])


def test_linear4_empty_and_errors(oracle_lib):
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    g = np.random.default_rng(13)
    R = rel(g, 50, 10, 5)
    for args in [(E, R, R, R), (R, E, R, R), (R, R, E, R), (R, R, R, E)]:
        assert oracle.linear4(*args, oracle.COUNT)["total"] == 0
    bad = (np.array([10], np.int32), np.array([0], np.int32))
    assert oracle.linear4(bad, R, R, R, oracle.GROUP_BY_A, a_domain=10, check=False)["rc"] == 2
