"""Seeded synthetic inputs for the 3-way join workloads.

This module produces data only: int32 column pairs shaped like the
workloads of the paper's evaluation (uniform join keys, Section 1.2's
no-skew assumption; friends relations of a social graph, Examples 1-4 and
Section 6.4).  It contains none of the join arithmetic, so that both the
CPU oracle and the CUDA path can consume the same inputs without sharing
any part of the method.

Every generator is deterministic in its ``seed`` (numpy PCG64).

Workload recipes (sizes as in the headline configurations):

* ``linear_uniform``: R(A,B), S(B,C), T(C,D) of 2^16 tuples each, A and D
  uniform in [0, 2^20), B and C uniform in [0, 2^12).
* ``chung_lu_directed``: a directed power-law "friends" relation F(src,dst)
  on 2^20 vertices.  Vertex weights follow a rank-Zipf law
  w_r = min(cap, c * r^-s) (s = 1.1, cap = 4096) with c chosen by bisection
  so that the mean weight is 32.  Sources are drawn with probability
  proportional to the out-weights and destinations proportional to the
  in-weights, with independent random rank->id permutations for the two
  sides; self loops and duplicate edges are dropped (a friends relation is
  a set).  Edges come out sorted by (src, dst), i.e. in adjacency order.
* ``chung_lu_undirected``: the same weight law on 2^22 vertices with mean
  undirected degree 32; both endpoints are drawn from the same weights,
  self loops and duplicates are dropped and every edge is oriented a < b.
* ``star_schema``: the star join of Section 6 (a large fact relation with
  two small dimension relations, TPC-H's lineitem with orders and supplier):
  R(A,B) and T(C,D) of 2^20 tuples each whose join keys B and C are unique
  (a random permutation of [0, 2^20)), A and D uniform attributes in
  [0, 2^16); the fact relation S(B,C) of 2^26 tuples holds foreign keys
  drawn uniformly (or Zipf(1.0) through a bijection) from the dimension
  keys, sorted by B like lineitem is by orderkey.
* ``skewed_linear``: R(A,B), S(B,C), T(C,D) whose B column is Zipf(s) in
  both R and S through one shared key bijection (heavy keys join each other),
  the other columns uniform; the skewed inputs of Section 7's future work.
* ``batched_queries``: many small independent joins with log-uniform sizes
  and key domains, keys uniform or Zipf(1.0) (P(k) proportional to
  1/(k+1), then mapped through a bijection of the domain).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 0x1905133760000000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed) & ((1 << 64) - 1)))


def uniform_relation(n: int, x_domain: int, y_domain: int, seed: int):
    """n tuples (x, y) with x ~ U[0, x_domain), y ~ U[0, y_domain), int32."""
    g = _rng(seed)
    x = g.integers(0, x_domain, size=n, dtype=np.int64).astype(np.int32)
    y = g.integers(0, y_domain, size=n, dtype=np.int64).astype(np.int32)
    return x, y


def linear_uniform(n: int = 1 << 16, ad: int = 1 << 20, bd: int = 1 << 12,
                   cd: int = 1 << 12, dd: int = 1 << 20, seed: int = SEED_BASE + 0):
    """R(A,B), S(B,C), T(C,D) with uniform keys (each relation its own stream)."""
    R = uniform_relation(n, ad, bd, seed * 3 + 1)
    S = uniform_relation(n, bd, cd, seed * 3 + 2)
    T = uniform_relation(n, cd, dd, seed * 3 + 3)
    return R, S, T


def zipf_rank_weights(n: int, mean: float, s: float = 1.1, cap: float = 4096.0):
    """Rank-Zipf weights w_r = min(cap, c r^-s), c set so that mean(w) = mean."""
    r = np.arange(1, n + 1, dtype=np.float64)
    base = r ** (-s)

    def mean_for(c):
        return float(np.minimum(cap, c * base).mean())

    lo, hi = 1e-9, 1e15
    for _ in range(90):
        mid = math.sqrt(lo * hi)
        if mean_for(mid) < mean:
            lo = mid
        else:
            hi = mid
    return np.minimum(cap, hi * base)


def _sample_by_weight(g: np.random.Generator, w: np.ndarray, m: int) -> np.ndarray:
    """m i.i.d. draws of an index with P(i) proportional to w[i].

    Drawn as multinomial counts followed by a uniform shuffle, which has the
    same distribution as m independent categorical draws.
    """
    p = np.asarray(w, dtype=np.float64)
    p = p / p.sum()
    counts = g.multinomial(m, p)
    idx = np.repeat(np.arange(len(p), dtype=np.int64), counts)
    g.shuffle(idx)
    return idx


def _sorted_distinct(code: np.ndarray) -> np.ndarray:
    code = np.sort(code)
    if code.size == 0:
        return code
    keep = np.empty(code.size, dtype=bool)
    keep[0] = True
    np.not_equal(code[1:], code[:-1], out=keep[1:])
    return code[keep]


def chung_lu_directed(n_vertices: int = 1 << 20, mean_degree: float = 32.0,
                      s: float = 1.1, cap: float = 4096.0,
                      seed: int = SEED_BASE + 1):
    """Directed power-law edge list (src, dst), deduplicated, no self loops."""
    g = _rng(seed)
    w = zipf_rank_weights(n_vertices, mean_degree, s, cap)
    perm_out = g.permutation(n_vertices).astype(np.int64)
    perm_in = g.permutation(n_vertices).astype(np.int64)
    m = int(round(n_vertices * mean_degree))
    src = perm_out[_sample_by_weight(g, w, m)]
    dst = perm_in[_sample_by_weight(g, w, m)]
    keep = src != dst
    code = _sorted_distinct(src[keep] * n_vertices + dst[keep])
    return (code // n_vertices).astype(np.int32), (code % n_vertices).astype(np.int32)


def chung_lu_undirected(n_vertices: int = 1 << 22, mean_degree: float = 32.0,
                        s: float = 1.1, cap: float = 4096.0,
                        seed: int = SEED_BASE + 2):
    """Undirected power-law edge set, each edge once as (a, b) with a < b."""
    g = _rng(seed)
    w = zipf_rank_weights(n_vertices, mean_degree, s, cap)
    perm = g.permutation(n_vertices).astype(np.int64)
    m = int(round(n_vertices * mean_degree / 2))
    u = perm[_sample_by_weight(g, w, m)]
    v = perm[_sample_by_weight(g, w, m)]
    keep = u != v
    lo = np.minimum(u[keep], v[keep])
    hi = np.maximum(u[keep], v[keep])
    code = _sorted_distinct(lo * n_vertices + hi)
    return (code // n_vertices).astype(np.int32), (code % n_vertices).astype(np.int32)


def triangle_relations(a: np.ndarray, b: np.ndarray):
    """R = S = E (a<b) and T = the reversed edges (c, a) with c > a.

    With both ends of every edge oriented low->high, the cyclic join
    R(A,B) S(B,C) T(C,A) needs T's tuples as (high, low): a triangle
    x < y < z then appears exactly once as (a,b,c) = (x,y,z).
    """
    return (a, b), (a, b), (b, a)


# ----------------------------------------------------------------------------
# Batched workload
# ----------------------------------------------------------------------------

@dataclass
class Query:
    kind: str                 # "linear" or "cyclic"
    R: tuple
    S: tuple
    T: tuple
    domains: tuple            # (A, B, C) or (A, B, C, D)
    zipf: bool


def _log_uniform_int(g, lo: int, hi: int) -> int:
    return int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))


_HARMONIC = {}


def _harmonic(s: float, size: int = 1 << 20) -> np.ndarray:
    """Cumulative weights H[k] = sum_{i<=k} (i+1)^-s for k < size (cached per s)."""
    key = round(float(s), 6)
    h = _HARMONIC.get(key)
    if h is None or len(h) < size:
        h = np.cumsum(np.power(np.arange(1, size + 1, dtype=np.float64), -s))
        _HARMONIC[key] = h
    return h


def _keys(g, n: int, domain: int, zipf: bool, s: float = 1.0) -> np.ndarray:
    if not zipf:
        return g.integers(0, domain, size=n, dtype=np.int64).astype(np.int32)
    # exact inverse CDF of P(k) proportional to (k+1)^-s on [0, domain)
    H = _harmonic(s, max(domain, 1 << 20))[:domain]
    # (searching sorted draws and shuffling the result gives the same i.i.d.
    # sample faster)
    k = np.searchsorted(H, np.sort(g.random(n)) * H[-1], side="right")
    g.shuffle(k)
    k = np.minimum(k, domain - 1).astype(np.int64)
    # bijection of [0, domain): k -> (k * mult + off) mod domain, gcd(mult, domain) = 1
    while True:
        mult = int(g.integers(1, max(2, domain)))
        if math.gcd(mult, domain) == 1:
            break
    off = int(g.integers(0, domain))
    return ((k * mult + off) % domain).astype(np.int32)


def skewed_linear(n: int = 1 << 22, s: float = 1.5, b_domain: int = 1 << 20,
                  c_domain: int = 1 << 22, a_domain: int = 1 << 20, seed: int = SEED_BASE + 6):
    """R(A,B), S(B,C), T(C,D) of n tuples each whose join column B is Zipf(s)
    in both R and S through one shared bijection of [0, b_domain) (so the
    heavy keys of R and S are the same keys); A, C, D uniform.  Stands in for
    the skewed inputs the paper leaves to future work."""
    g = _rng(seed)
    H = _harmonic(s, max(b_domain, 1 << 20))[:b_domain]
    while True:
        mult = int(g.integers(1, max(2, b_domain)))
        if math.gcd(mult, b_domain) == 1:
            break
    off = int(g.integers(0, b_domain))

    def zipf_b():
        k = np.searchsorted(H, g.random(n) * H[-1], side="right")
        k = np.minimum(k, b_domain - 1).astype(np.int64)
        return ((k * mult + off) % b_domain).astype(np.int32)

    R = (g.integers(0, a_domain, n, dtype=np.int64).astype(np.int32), zipf_b())
    S = (zipf_b(), g.integers(0, c_domain, n, dtype=np.int64).astype(np.int32))
    T = (g.integers(0, c_domain, n, dtype=np.int64).astype(np.int32),
         g.integers(0, a_domain, n, dtype=np.int64).astype(np.int32))
    return R, S, T


def star_schema(n_fact: int = 1 << 26, n_dim: int = 1 << 20, attr_domain: int = 1 << 16,
                zipf: bool = False, sorted_fact: bool = True, seed: int = SEED_BASE + 5):
    """(R, S, T) of a star join: dimensions R(A,B), T(C,D) with unique keys,
    fact S(B,C) of foreign keys into them (every S tuple joins exactly one R
    and one T tuple)."""
    g = _rng(seed)
    rb = g.permutation(n_dim).astype(np.int32)
    ra = g.integers(0, attr_domain, size=n_dim, dtype=np.int64).astype(np.int32)
    tc = g.permutation(n_dim).astype(np.int32)
    td = g.integers(0, attr_domain, size=n_dim, dtype=np.int64).astype(np.int32)
    sb = _keys(g, n_fact, n_dim, zipf)
    sc = _keys(g, n_fact, n_dim, zipf)
    if sorted_fact:
        o = np.argsort(sb, kind="stable")
        sb, sc = sb[o], sc[o]
    return (ra, rb), (np.ascontiguousarray(sb), np.ascontiguousarray(sc)), (tc, td)


def random_query(g, kind: str, size_lo: int = 1 << 8, size_hi: int = 1 << 18,
                 dom_lo: int = 1 << 6, dom_hi: int = 1 << 20, zipf=None,
                 zipf_s: float = 1.0) -> Query:
    if zipf is None:
        zipf = bool(g.integers(0, 2))
    nR, nS, nT = (_log_uniform_int(g, size_lo, size_hi) for _ in range(3))
    if kind == "linear":
        dA, dB, dC, dD = (_log_uniform_int(g, dom_lo, dom_hi) for _ in range(4))
        R = (_keys(g, nR, dA, zipf, zipf_s), _keys(g, nR, dB, zipf, zipf_s))
        S = (_keys(g, nS, dB, zipf, zipf_s), _keys(g, nS, dC, zipf, zipf_s))
        T = (_keys(g, nT, dC, zipf, zipf_s), _keys(g, nT, dD, zipf, zipf_s))
        doms = (dA, dB, dC, dD)
    else:
        dA, dB, dC = (_log_uniform_int(g, dom_lo, dom_hi) for _ in range(3))
        R = (_keys(g, nR, dA, zipf, zipf_s), _keys(g, nR, dB, zipf, zipf_s))
        S = (_keys(g, nS, dB, zipf, zipf_s), _keys(g, nS, dC, zipf, zipf_s))
        T = (_keys(g, nT, dC, zipf, zipf_s), _keys(g, nT, dA, zipf, zipf_s))
        doms = (dA, dB, dC)
    return Query(kind, R, S, T, doms, zipf)


def batched_queries(n_queries: int = 4096, seed: int = SEED_BASE + 3, **kw):
    """n_queries independent joins, linear and cyclic alternating 50/50."""
    g = _rng(seed)
    return [random_query(g, "linear" if q % 2 == 0 else "cyclic", **kw)
            for q in range(n_queries)]
