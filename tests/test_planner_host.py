"""Host logic of the learned planner (CPU): the share scale applies to the
partitioned plan, and the plan-time bookkeeping picks the right entries."""
import math

from paper_1905_13376_gb300 import binding, planner


class FakeCtx:
    """plan_shares of the library: (1,1,1) for the linear aggregates, H(B)
    buckets for row output; cyclic cube shares."""

    def __init__(self):
        self.modes = []

    def plan_shares(self, kind, R, S, T, mode=binding.MWJ_COUNT):
        self.modes.append(mode)
        if kind == binding.MWJ_LINEAR:
            return (1, 1, 1) if mode != binding.MWJ_MATERIALIZE else (1024, 1, 1)
        return (64, 32, 16)


def test_linear_scale_applies_to_the_partitioned_plan():
    ctx = FakeCtx()
    got = {k: planner.scaled_shares(ctx, binding.MWJ_LINEAR, None, None, None, k) for k in planner.SCALES}
    assert got == {-1: (512, 1, 1), 0: (1024, 1, 1), 1: (2048, 1, 1)}
    assert set(ctx.modes) == {binding.MWJ_MATERIALIZE}


def test_cyclic_scale_keeps_every_face_of_the_cube_in_bounds():
    ctx = FakeCtx()
    for k in planner.SCALES:
        sh = planner.scaled_shares(ctx, binding.MWJ_CYCLIC, None, None, None, k)
        assert min(sh) >= 1
        assert sh[0] * sh[1] <= 32768 and sh[1] * sh[2] <= 32768 and sh[2] * sh[0] <= 32768
    assert planner.scaled_shares(ctx, binding.MWJ_CYCLIC, None, None, None, 0) == (64, 32, 16)


def test_plan_time_and_best_time():
    t = {("mw", -1): 30.0, ("mw", 0): 20.0, ("mw", 1): 25.0, "cascade": None}
    assert planner.plan_time(t, (False, 0)) == 20.0
    assert planner.plan_time(t, (True, 0)) == math.inf    # cascade not run: never chosen as best
    assert planner.best_time(t) == 20.0
    t["cascade"] = 12.5
    assert planner.plan_time(t, (True, 1)) == 12.5 and planner.best_time(t) == 12.5
