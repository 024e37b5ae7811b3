"""The library's cost model (mwj_cost_model, called through the C ABI on the
host; no GPU work) against the paper's tuple counts in oracle/costmodel.py.
With a tiny HBM bandwidth every phase is bandwidth-bound, so differences
between two instances isolate the byte terms: the cascade writes its
intermediate and reads it back (Example 3), the linear 3-way join reads R and
S once while T's table is held whole (Section 4.2), and the cube tiling reads
|R| + 2 sqrt(|R||S||T|/M) tuples at the optimal share (Section 5.2)."""
import numpy as np
import pytest

from oracle import costmodel as cm
from paper_1905_13376_gb300 import binding

BW = 1e-3          # GB/s: bandwidth terms dominate every other term
BPS = BW * 1e9     # bytes/s


def feats(nR, nS, nT, nI, cyclic=False, dB=1e3, dC=1e3):
    f = np.zeros(24, np.float32)
    f[0], f[1], f[2] = (np.log2(1.0 + v) for v in (nR, nS, nT))
    f[4], f[5] = np.log2(1.0 + dB), np.log2(1.0 + dC)
    f[7] = 1.0 if cyclic else 0.0
    f[8] = np.log2(1.0 + nI)
    return f


def seconds(f):
    return [2.0 ** v for v in binding.cost_model(f, BW)]


def sizes(f):
    """The sizes the model sees (the features are float32 logs)."""
    return [2.0 ** float(np.float32(v)) - 1.0 for v in (f[0], f[1], f[2], f[8])]


@pytest.mark.parametrize("cyclic", [False, True])
def test_cascade_moves_the_intermediate_twice(cyclic):
    f1, f2 = feats(1e5, 2e5, 3e5, 1e6, cyclic), feats(1e5, 2e5, 3e5, 4e7, cyclic)
    dI = sizes(f2)[3] - sizes(f1)[3]
    got = seconds(f2)[0] - seconds(f1)[0]
    # Example 3: the cascade writes I and reads it back (12 bytes per row each
    # way); the cyclic cascade also writes I once more, grouped by (c, a) for
    # the second join (8 bytes per row)
    want = (12.0 * cm.cascade_tuples_moved(dI) + (8.0 * dI if cyclic else 0.0)) / BPS
    assert got == pytest.approx(want, rel=1e-6)


def test_linear_reads_R_and_S_once_with_T_held_whole():
    base = feats(1e5, 2e5, 3e5, 1e6)
    more = feats(7e5, 9e5, 3e5, 1e6)
    (r1, s1, t1, _), (r2, s2, t2, _) = sizes(base), sizes(more)
    M = float("inf")   # T's table held whole on chip: the |R||T|/M term vanishes
    dreads = cm.linear_tuples_read(r2, s2, t2, M) - cm.linear_tuples_read(r1, s1, t1, M)
    got = seconds(more)[1] - seconds(base)[1]
    assert got == pytest.approx(8.0 * dreads / BPS, rel=1e-6)
    # the partitioned alternative also writes and reads R and S once more
    got_alt = seconds(more)[2] - seconds(base)[2]
    assert got_alt == pytest.approx(24.0 * dreads / BPS, rel=1e-6)


def test_cyclic_cube_reads_the_optimal_cost():
    a = feats(3e5, 2e5, 5e5, 1.0, cyclic=True)
    b = feats(3e5, 8e5, 5e5, 1.0, cyclic=True)
    (r1, s1, t1, _), (r2, s2, t2, _) = sizes(a), sizes(b)
    M = 1024.0
    dreads = cm.cyclic_optimal_cost(r2, s2, t2, M) - cm.cyclic_optimal_cost(r1, s1, t1, M)
    got = seconds(b)[2] - seconds(a)[2]
    # partitioning S once more (20 bytes per tuple) plus the tile reads
    want = (20.0 * (s2 - s1) + 8.0 * dreads) / BPS
    assert got == pytest.approx(want, rel=1e-4)


def test_plans_ordered_by_intermediate_size():
    """Far below the inputs the cascade is the cheaper or close plan; far above
    it loses to the 3-way join (the paper's crossover argument)."""
    for cyclic in (False, True):
        small = binding.cost_model(feats(1e6, 1e6, 1e6, 1e4, cyclic), 6792.1)
        big = binding.cost_model(feats(1e6, 1e6, 1e6, 1e10, cyclic), 6792.1)
        assert big[0] > small[0] + 5
        assert big[0] > big[1]
