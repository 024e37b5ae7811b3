"""Exact GROUP BY A of the linear join summed in factorised order (numpy,
int64), for full-size checks where the oracle's walk over every (R, S) pair
is too slow.  Pinned against the oracle in tests/test_oracle.py."""
import numpy as np


def factorised_group_by(R, S, T, a_domain):
    """cnt(a) = sum over (a,b) in R of w(b), w(b) = sum over (b,c) in S of
    deg_T(c): the GROUP BY A definition summed in another order, in exact
    int64 (the oracle walks every (R, S) pair, too slow at |R|x|S| ~ 1e12;
    tests/test_oracle.py pins this form against the oracle)."""
    off = np.int64(1) << 31
    ck, cc = np.unique(T[0], return_counts=True)
    keys_t = ck.astype(np.int64)
    # deg_T(c) for every S tuple
    pos = np.searchsorted(keys_t, S[1].astype(np.int64))
    pos = np.minimum(pos, len(keys_t) - 1)
    dS = np.where(keys_t[pos] == S[1], cc[pos], 0).astype(np.int64)
    bk, inv = np.unique(S[0].astype(np.int64) + off, return_inverse=True)
    w = np.zeros(len(bk), dtype=np.int64)
    np.add.at(w, inv, dS)
    pr = np.searchsorted(bk, R[1].astype(np.int64) + off)
    pr = np.minimum(pr, len(bk) - 1)
    wR = np.where(bk[pr] == R[1].astype(np.int64) + off, w[pr], 0)
    cnt = np.zeros(a_domain, dtype=np.int64)
    np.add.at(cnt, R[0].astype(np.int64), wR)
    return int(cnt.sum()), cnt
