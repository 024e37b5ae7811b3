"""Pins of the CPU oracle to things other than itself (no GPU needed).

Every check here uses an independent route to the same number: pure-Python
nested loops over the definition, numpy closed forms, graph identities
(trace(A^3)/6, C(n,3)), constructed special cases and invariants.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import COUNT, GROUP_BY_A, MATERIALIZE
from paper_1905_13376_gb300 import datagen

U64 = 1 << 64


def brute_linear(R, S, T):
    rows = []
    for a, b in zip(*R):
        for b2, c in zip(*S):
            if b2 != b:
                continue
            for c2, d in zip(*T):
                if c2 == c:
                    rows.append((int(a), int(b), int(c), int(d)))
    return sorted(rows)


def brute_cyclic(R, S, T):
    rows = []
    for a, b in zip(*R):
        for b2, c in zip(*S):
            if b2 != b:
                continue
            for c2, a2 in zip(*T):
                if c2 == c and a2 == a:
                    rows.append((int(a), int(b), int(c)))
    return sorted(rows)


def rand_rel(g, n, dx, dy, lo=0):
    return (g.integers(lo, dx, n).astype(np.int32), g.integers(lo, dy, n).astype(np.int32))


def group_by_from_rows(rows, a_domain):
    cnt = np.zeros(a_domain, dtype=np.int64)
    for r in rows:
        cnt[r[0]] += 1
    return cnt


@pytest.mark.parametrize("seed", range(12))
def test_linear_vs_brute_force(oracle_lib, seed):
    g = np.random.default_rng(seed)
    dom = int(g.integers(1, 6))
    nR, nS, nT = (int(g.integers(0, 30)) for _ in range(3))
    R = rand_rel(g, nR, 8, dom)
    S = rand_rel(g, nS, dom, dom)
    T = rand_rel(g, nT, dom, 9)
    rows = brute_linear(R, S, T)
    out = oracle.linear(R, S, T, COUNT)
    assert out["total"] == len(rows)
    gb = oracle.linear(R, S, T, GROUP_BY_A, a_domain=8)
    assert np.array_equal(gb["counts"], group_by_from_rows(rows, 8))
    assert gb["total"] == len(rows)
    mat = oracle.linear(R, S, T, MATERIALIZE, capacity=len(rows) + 3)
    assert mat["n_rows"] == len(rows)
    assert [tuple(r) for r in mat["rows"].tolist()] == rows


@pytest.mark.parametrize("seed", range(12))
def test_cyclic_vs_brute_force(oracle_lib, seed):
    g = np.random.default_rng(100 + seed)
    da, db, dc = (int(g.integers(1, 5)) for _ in range(3))
    nR, nS, nT = (int(g.integers(0, 30)) for _ in range(3))
    R = rand_rel(g, nR, da, db)
    S = rand_rel(g, nS, db, dc)
    T = rand_rel(g, nT, dc, da)
    rows = brute_cyclic(R, S, T)
    assert oracle.cyclic(R, S, T, COUNT)["total"] == len(rows)
    gb = oracle.cyclic(R, S, T, GROUP_BY_A, a_domain=da)
    assert np.array_equal(gb["counts"], group_by_from_rows(rows, da))
    mat = oracle.cyclic(R, S, T, MATERIALIZE, capacity=len(rows))
    assert [tuple(r) for r in mat["rows"].tolist()] == rows


def test_linear_brute_force_negative_and_extreme_keys(oracle_lib):
    vals = np.array([-2**31, 2**31 - 1, -1, 0, 7], dtype=np.int32)
    g = np.random.default_rng(5)
    R = (g.integers(0, 6, 25).astype(np.int32), vals[g.integers(0, 5, 25)])
    S = (vals[g.integers(0, 5, 25)], vals[g.integers(0, 5, 25)])
    T = (vals[g.integers(0, 5, 25)], g.integers(-5, 5, 25).astype(np.int32))
    rows = brute_linear(R, S, T)
    assert oracle.linear(R, S, T)["total"] == len(rows)
    mat = oracle.linear(R, S, T, MATERIALIZE)
    assert [tuple(r) for r in mat["rows"].tolist()] == rows
    Tc = (vals[g.integers(0, 5, 25)], R[0][g.integers(0, 25, 25)])
    rows_c = brute_cyclic(R, S, Tc)
    assert oracle.cyclic(R, S, Tc)["total"] == len(rows_c)


def _dense_ids(*cols):
    allv = np.concatenate(cols)
    uniq, inv = np.unique(allv, return_inverse=True)
    out, p = [], 0
    for c in cols:
        out.append(inv[p:p + len(c)])
        p += len(c)
    return len(uniq), out


def closed_form_linear(R, S, T):
    """sum_{(b,c) in S} deg_R(b) deg_T(c) with numpy histograms (mod 2^64)."""
    nb, (Rb, Sb) = _dense_ids(R[1], S[0])
    nc, (Sc, Tc) = _dense_ids(S[1], T[0])
    degR = np.bincount(Rb, minlength=nb).astype(np.uint64)
    degT = np.bincount(Tc, minlength=nc).astype(np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(degR[Sb] * degT[Sc], dtype=np.uint64))


def factorised_group_by(R, S, T, a_domain):
    """cnt[a] = sum_{(a,b) in R} w[b],  w[b] = sum_{(b,c) in S} deg_T(c)."""
    nb, (Rb, Sb) = _dense_ids(R[1], S[0])
    nc, (Sc, Tc) = _dense_ids(S[1], T[0])
    degT = np.bincount(Tc, minlength=nc).astype(np.uint64)
    w = np.zeros(nb, dtype=np.uint64)
    np.add.at(w, Sb, degT[Sc])
    cnt = np.zeros(a_domain, dtype=np.uint64)
    np.add.at(cnt, R[0].astype(np.int64), w[Rb])
    return cnt.view(np.int64)


def test_linear_closed_form_uniform_config(oracle_lib):
    R, S, T = datagen.linear_uniform()
    out = oracle.linear(R, S, T, GROUP_BY_A, a_domain=1 << 20)
    assert out["total"] == closed_form_linear(R, S, T)
    assert np.array_equal(out["counts"], factorised_group_by(R, S, T, 1 << 20))
    assert int(out["counts"].sum()) == out["total"]
    # 2^16 S tuples, each matching ~16 R and ~16 T tuples
    assert 0.9 * 2**24 < out["total"] < 1.1 * 2**24


def test_linear_closed_form_skewed(oracle_lib):
    g = np.random.default_rng(9)
    q = datagen.random_query(g, "linear", size_lo=3000, size_hi=6000, dom_lo=50,
                             dom_hi=400, zipf=True, zipf_s=1.3)
    out = oracle.linear(q.R, q.S, q.T, GROUP_BY_A, a_domain=q.domains[0])
    assert out["total"] == closed_form_linear(q.R, q.S, q.T)
    assert np.array_equal(out["counts"], factorised_group_by(q.R, q.S, q.T, q.domains[0]))


def _triangles_by_trace(n, edges):
    A = np.zeros((n, n), dtype=np.int64)
    for u, v in edges:
        A[u, v] = A[v, u] = 1
    return int(np.trace(A @ A @ A)) // 6


def _oriented(edges):
    a = np.array([min(u, v) for u, v in edges], dtype=np.int32)
    b = np.array([max(u, v) for u, v in edges], dtype=np.int32)
    return datagen.triangle_relations(a, b)


@pytest.mark.parametrize("seed", range(6))
def test_triangles_trace(oracle_lib, seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(5, 64))
    p = float(g.uniform(0.05, 0.6))
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if g.random() < p]
    R, S, T = _oriented(edges)
    assert oracle.cyclic(R, S, T)["total"] == _triangles_by_trace(n, edges)


@pytest.mark.parametrize("n", [3, 4, 10, 57, 200])
def test_triangles_complete_graph(oracle_lib, n):
    edges = list(itertools.combinations(range(n), 2))
    R, S, T = _oriented(edges)
    assert oracle.cyclic(R, S, T)["total"] == math.comb(n, 3)


def test_single_triangle_and_orientation(oracle_lib):
    R, S, T = _oriented([(0, 1), (1, 2), (0, 2)])
    out = oracle.cyclic(R, S, T, MATERIALIZE)
    assert out["rows"].tolist() == [[0, 1, 2]]
    # without reversing T the oriented join is empty (a < b < c < a impossible)
    assert oracle.cyclic(R, S, R)["total"] == 0


def test_single_key_everywhere(oracle_lib):
    nR, nS, nT = 37, 11, 23
    R = (np.arange(nR, dtype=np.int32), np.full(nR, 5, np.int32))
    S = (np.full(nS, 5, np.int32), np.full(nS, -9, np.int32))
    T = (np.full(nT, -9, np.int32), np.arange(nT, dtype=np.int32))
    assert oracle.linear(R, S, T)["total"] == nR * nS * nT
    Rc = (np.zeros(nR, np.int32), np.zeros(nR, np.int32))
    Sc = (np.zeros(nS, np.int32), np.zeros(nS, np.int32))
    Tc = (np.zeros(nT, np.int32), np.zeros(nT, np.int32))
    assert oracle.cyclic(Rc, Sc, Tc)["total"] == nR * nS * nT


def test_disjoint_and_empty(oracle_lib):
    R = (np.arange(10, dtype=np.int32), np.arange(10, dtype=np.int32))
    S = (np.arange(10, 20, dtype=np.int32), np.arange(10, dtype=np.int32))
    assert oracle.linear(R, S, R)["total"] == 0
    E = (np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert oracle.linear(E, S, R)["total"] == 0
    assert oracle.cyclic(R, E, R)["total"] == 0
    out = oracle.linear(R, R, R, MATERIALIZE, capacity=0, check=False)
    assert out["rc"] == 3 and out["n_rows"] == 10


def test_bag_semantics_duplicates_count(oracle_lib):
    g = np.random.default_rng(3)
    R = rand_rel(g, 20, 4, 3)
    S = rand_rel(g, 20, 3, 3)
    T = rand_rel(g, 20, 3, 4)
    base = oracle.linear(R, S, T)["total"]
    R2 = (np.concatenate([R[0], R[0]]), np.concatenate([R[1], R[1]]))
    assert oracle.linear(R2, S, T)["total"] == 2 * base
    T3 = (np.concatenate([T[0]] * 3), np.concatenate([T[1]] * 3))
    assert oracle.linear(R, S, T3)["total"] == 3 * base


def test_domain_and_capacity_errors(oracle_lib):
    R = (np.array([0, 5], np.int32), np.array([1, 1], np.int32))
    S = (np.array([1], np.int32), np.array([2], np.int32))
    T = (np.array([2, 2, 2], np.int32), np.array([0, 1, 2], np.int32))
    out = oracle.linear(R, S, T, GROUP_BY_A, a_domain=5, check=False)
    assert out["rc"] == 2
    out = oracle.linear(R, S, T, MATERIALIZE, capacity=4, check=False)
    assert out["rc"] == 3 and out["n_rows"] == 6


def test_count_wraps_mod_2_64(oracle_lib):
    # one key everywhere: the count |R||S||T| exceeds 2^64 and must wrap
    nR, nS, nT = 1 << 22, 1 << 21, (1 << 21) + 3
    R = (np.zeros(nR, np.int32), np.zeros(nR, np.int32))
    S = (np.zeros(nS, np.int32), np.zeros(nS, np.int32))
    T = (np.zeros(nT, np.int32), np.zeros(nT, np.int32))
    want = (nR * nS * nT) % U64
    got = oracle.linear(R, S, T)["total"] % U64
    assert got == want


def test_binary_count(oracle_lib):
    g = np.random.default_rng(4)
    R = rand_rel(g, 50, 5, 4)
    S = rand_rel(g, 40, 4, 5)
    brute = sum(1 for b in R[1] for b2 in S[0] if b == b2)
    assert oracle.binary_count(R, S) == brute


def test_factorised_group_by_matches_oracle(oracle_lib):
    """The factorised form the full-size skew test uses, against the oracle
    on skewed inputs (heavy keys shared by R and S) and on the uniform config."""
    from factorised import factorised_group_by
    from paper_1905_13376_gb300 import datagen
    for R, S, T, dom in [
        datagen.skewed_linear(n=1 << 14, s=1.3, b_domain=1 << 11, c_domain=1 << 10,
                              a_domain=1 << 9, seed=77) + (1 << 9,),
        datagen.linear_uniform(n=4000, ad=1 << 9, bd=64, cd=64, dd=100, seed=5) + (1 << 9,),
    ]:
        want = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=dom)
        total, cnt = factorised_group_by(R, S, T, dom)
        assert total == want["total"]
        assert np.array_equal(cnt, want["counts"])
