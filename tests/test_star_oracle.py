"""The oracle on star-join inputs (Section 6's star 3-way join: a fact
relation S(B,C) of foreign keys into two dimension relations with unique
keys).  Every S tuple then joins exactly one R tuple and one T tuple, so

    COUNT(*)            = |S|
    COUNT(*) GROUP BY A = for each a, the number of S tuples whose b is the
                          key of an R tuple with attribute a

which pins the oracle (and the generator's star shape) without re-running
any join."""
import numpy as np
import pytest

import oracle
from paper_1905_13376_gb300 import datagen


@pytest.mark.parametrize("zipf", [False, True])
def test_star_schema_closed_form(oracle_lib, zipf):
    R, S, T = datagen.star_schema(n_fact=1 << 16, n_dim=1 << 12, attr_domain=1 << 8, zipf=zipf,
                                  seed=datagen.SEED_BASE + 50 + int(zipf))
    ra, rb = R
    sb, sc = S
    # dimension keys are unique and every foreign key exists
    assert len(np.unique(rb)) == len(rb) and len(np.unique(T[0])) == len(T[0])
    assert np.isin(sb, rb).all() and np.isin(sc, T[0]).all()
    inv = np.empty(len(rb), dtype=np.int64)
    inv[rb] = np.arange(len(rb))
    want = np.bincount(ra[inv[sb]], minlength=1 << 8)
    got = oracle.linear(R, S, T, oracle.GROUP_BY_A, a_domain=1 << 8)
    assert got["total"] == len(sb)
    assert np.array_equal(got["counts"], want)


def test_star_schema_missing_foreign_keys(oracle_lib):
    """S tuples whose b or c has no dimension tuple join nothing."""
    R, S, T = datagen.star_schema(n_fact=4096, n_dim=256, attr_domain=16,
                                  seed=datagen.SEED_BASE + 52)
    keep = R[1] % 3 != 0      # drop a third of R's keys
    R2 = (R[0][keep], R[1][keep])
    keepT = T[0] % 5 != 0     # and a fifth of T's
    T2 = (T[0][keepT], T[1][keepT])
    want = int(np.sum((S[0] % 3 != 0) & (S[1] % 5 != 0)))
    assert oracle.linear(R2, S, T2, oracle.COUNT)["total"] == want
