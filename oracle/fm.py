"""Flajolet-Martin sketches of the friends-of-friends-of-friends sets --
TEST INFRASTRUCTURE ONLY (tests, smoke check and the CPU baseline may use it;
the CUDA path never does).

Section 4.1's footnote and Example 1 estimate, for every person A, the number
of distinct D reachable as (a,b) in R, (b,c) in S, (c,d) in T, with the
Flajolet-Martin algorithm instead of an exact distinct count.  Here

    D(a) = { d : (a,b) in R, (b,c) in S, (c,d) in T }          (a set)

and its sketch is Flajolet and Martin's probabilistic counting with
stochastic averaging (PCSA; "Probabilistic counting algorithms for data base
applications", 1985) with M = 16 bitmaps of 32 bits:

    h      = fmix32(d xor SEED)   (MurmurHash3's 32-bit finaliser)
    bitmap = h mod M,  bit = rho(h div M)  (index of the lowest 1 bit, 0-based;
                                            27 when h div M is 0)
    sketch(a) = OR over d in D(a) of that bit

so the sketch of a union is the OR of the sketches, which is what lets the
join carry sketches along the chain exactly as it carries counts.  The
estimate is (M / PHI) * 2^(mean over bitmaps of R_j), R_j the index of the
lowest 0 bit of bitmap j, PHI = 0.77351 (PCSA's correction factor); its
relative standard error is about 0.78 / sqrt(M).

Everything here follows those definitions directly: D(a) is built as an
explicit set from grouped lists, and the sketch is the OR of the bits of its
members.
"""
from __future__ import annotations

import numpy as np

M = 16
SEED = 0x5BD1E995
PHI = 0.77351
MASK32 = 0xFFFFFFFF


def fmix32(x: int) -> int:
    """MurmurHash3's 32-bit finalisation mix (Appleby's published constants)."""
    x &= MASK32
    x ^= x >> 16
    x = (x * 0x85EBCA6B) & MASK32
    x ^= x >> 13
    x = (x * 0xC2B2AE35) & MASK32
    x ^= x >> 16
    return x


def bit_of(d: int) -> tuple[int, int]:
    """(bitmap, bit) that value d sets."""
    h = fmix32((int(d) & MASK32) ^ SEED)
    j = h % M
    q = h // M
    if q == 0:
        return j, 27
    r = (q & -q).bit_length() - 1
    return j, r


def sketch_of(values) -> np.ndarray:
    sk = np.zeros(M, dtype=np.uint32)
    for d in set(int(v) for v in values):
        j, r = bit_of(d)
        sk[j] |= np.uint32(1 << r)
    return sk


def estimate(sk) -> float:
    """PCSA estimate from one sketch (M uint32 bitmaps)."""
    tot = 0
    for w in np.asarray(sk, dtype=np.uint64):
        w = int(w)
        r = 0
        while (w >> r) & 1:
            r += 1
        tot += r
    return (M / PHI) * 2.0 ** (tot / M)


def _groups(x, y):
    g = {}
    for a, b in zip(np.asarray(x).tolist(), np.asarray(y).tolist()):
        g.setdefault(a, []).append(b)
    return g


def fof3_sets(R, S, T, a_values):
    """D(a) for each a in a_values, as Python sets (R, S, T are (x, y) pairs)."""
    Rg, Sg, Tg = _groups(*R), _groups(*S), _groups(*T)
    out = {}
    for a in a_values:
        bs = set(Rg.get(int(a), ()))
        cs = set()
        for b in bs:
            cs.update(Sg.get(b, ()))
        ds = set()
        for c in cs:
            ds.update(Tg.get(c, ()))
        out[int(a)] = ds
    return out


def sketches(R, S, T, a_domain: int):
    """(a_domain, M) uint32 sketches and exact |D(a)| for every a."""
    D = fof3_sets(R, S, T, range(a_domain))
    sk = np.zeros((a_domain, M), dtype=np.uint32)
    n = np.zeros(a_domain, dtype=np.int64)
    for a, ds in D.items():
        sk[a] = sketch_of(ds)
        n[a] = len(ds)
    return sk, n


def _csr(x, y):
    """key -> values as (sorted unique keys, starts, values grouped by key)."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    o = np.argsort(x, kind="stable")
    keys, starts = np.unique(x[o], return_index=True)
    return keys, np.append(starts, len(x)), y[o]


def _expand(csr, vals):
    """The set of values reached from the keys `vals` through one relation."""
    keys, starts, out = csr
    vals = np.unique(np.asarray(vals, dtype=np.int64))
    p = np.searchsorted(keys, vals)
    inside = p < len(keys)
    p, vals = p[inside], vals[inside]
    p = p[keys[p] == vals]
    parts = [out[starts[i]:starts[i + 1]] for i in p]
    return np.unique(np.concatenate(parts)) if parts else np.zeros(0, np.int64)


def fof3_sets_csr(R, S, T, a_values):
    """D(a) for each a (numpy arrays), the same sets as fof3_sets, for
    relations too large for Python dictionaries."""
    Rc, Sc, Tc = _csr(*R), _csr(*S), _csr(*T)
    return {int(a): _expand(Tc, _expand(Sc, _expand(Rc, [a]))) for a in a_values}
