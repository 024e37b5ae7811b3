"""Host logic of the learned planner (CPU): which shares each plan uses, the
masked labels, and the regret bookkeeping of the evaluation."""
import math

import numpy as np
import pytest

from paper_1905_13376_gb300 import binding, planner


class FakeCtx:
    """plan_shares_alt of the library, recorded."""

    def __init__(self):
        self.calls = []

    def plan_shares_alt(self, kind, R, S, T):
        self.calls.append(kind)
        return (1024, 1, 1) if kind == binding.MWJ_LINEAR else (64, 32, 16)


def test_plan_shares_of_the_three_plans():
    ctx = FakeCtx()
    assert planner.plan_shares(ctx, binding.MWJ_LINEAR, None, None, None, 1) is None   # library default
    assert planner.plan_shares(ctx, binding.MWJ_LINEAR, None, None, None, 2) == (1024, 1, 1)
    assert planner.plan_shares(ctx, binding.MWJ_CYCLIC, None, None, None, 2) == (64, 32, 16)
    assert ctx.calls == [binding.MWJ_LINEAR, binding.MWJ_CYCLIC]
    with pytest.raises(ValueError):
        planner.plan_shares(ctx, binding.MWJ_LINEAR, None, None, None, 0)


def test_labels_mask_plans_that_were_not_run():
    Y, M = planner.labels([[None, 10.0, 20.0], [5.0, 8.0, 16.0]])
    assert M.tolist() == [[0, 1, 1], [1, 1, 1]]
    assert Y[1].tolist() == pytest.approx([math.log2(5), 3.0, 4.0])
    assert Y[0, 1] == pytest.approx(math.log2(10))


class FakePlanner:
    def __init__(self, picks):
        self.picks = picks

    def choose(self, F):
        return list(self.picks)


def feats(nR, nS, nT, nI):
    f = np.zeros(24, np.float32)
    f[0], f[1], f[2] = (np.log2(1.0 + v) for v in (nR, nS, nT))
    f[4] = f[5] = np.log2(1.0 + 1000)
    f[8] = np.log2(1.0 + nI)
    return f


def test_regret_against_the_best_measured_plan():
    F = np.stack([feats(1e4, 1e4, 1e4, 1e3), feats(1e4, 1e4, 1e4, 1e9), feats(1e4, 1e4, 1e4, 1e6)])
    times = [[30.0, 10.0, 15.0],      # default plan best
             [None, 50.0, 40.0],      # cascade not run; alternative best
             [100.0, 20.0, 25.0]]     # intermediate above the inputs, cascade runnable
    summary, res = planner.evaluate(FakePlanner([1, 1, 2]), F, times, sizes=[[1e4] * 3] * 3)
    assert res["learned"] == pytest.approx([0.0, 0.25, 0.25])
    assert res["default"] == pytest.approx([0.0, 0.25, 0.0])
    assert res["alt"] == pytest.approx([0.5, 0.0, 0.25])
    assert res["cascade"][1] == float("inf")
    assert summary["cascade"]["not_runnable"] == 1
    assert summary["learned"]["within_10pct"] == pytest.approx(1 / 3)
    big = summary["intermediate_above_inputs"]
    assert big["instances"] == 2 and big["cascade_not_runnable"] == 1
    assert big["learned_beats_cascade"] == 1.0
    assert big["geo_mean_speedup_over_cascade_runnable"] == pytest.approx(100.0 / 25.0)


def test_times_round_trip_through_the_saved_dataset():
    times = [[None, 1.5, 2.0], [3.0, 4.0, None]]
    assert planner._array_to_times(planner._times_to_array(times)) == times


def test_a_cascade_too_large_runs_as_the_3way_join():
    """A choice of the cascade whose estimated intermediate (feature 8 =
    log2(|R join S| + 1)) is above the limit runs as the 3-way join with the
    default shares, in plan_and_run and in the evaluation alike."""
    f = np.zeros(24, np.float32)
    f[8] = 31.0
    assert planner.runnable(0, f) == 1
    f[8] = 20.0
    assert planner.runnable(0, f) == 0
    assert planner.runnable(2, f) == 2 and planner.runnable(1, f) == 1
