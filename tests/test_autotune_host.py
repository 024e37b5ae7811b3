"""The batch autotuner's search on the host: a stand-in context records the
rules and launch shapes the tuner installs and a stand-in timer prices them,
so that the choice logic (one class at a time, the 3 % margin, the check on
the whole batch) is tested without a GPU."""
import json

import pytest
import torch

from paper_1905_13376_gb300 import autotune, binding

LIN, CYC = binding.MWJ_LINEAR, binding.MWJ_CYCLIC


class FakeCtx:
    def __init__(self):
        self.rules, self.launch = [], (0, 0)

    def batch_set_rules(self, rules):
        self.rules = [tuple(r) for r in rules]

    def batch_set_launch(self, a, b):
        self.launch = (a, b)


def rel(n):
    return (torch.zeros(n, dtype=torch.int32), torch.zeros(n, dtype=torch.int32))


def batch():
    """40 linear queries of 2^12 tuples (class (LIN, 12)) and 40 cyclic ones
    whose largest relation has 2^14 (class (CYC, 14))."""
    return ([(LIN, rel(1 << 12), rel(1 << 12), rel(1 << 12)) for _ in range(40)] +
            [(CYC, rel(1 << 14), rel(100), rel(100)) for _ in range(40)])


def priced(gains, whole_penalty=0.0):
    """A timer: 10 ms less each installed (rule or launch) gain; a launch of
    the whole batch (80 queries) pays whole_penalty for every installed rule."""
    def t(ctx, qs, reps):
        ms = 10.0
        for r in ctx.rules:
            ms -= gains.get(r, 0.0)
        ms -= gains.get(ctx.launch, 0.0)
        if len(qs) == 80:
            ms += whole_penalty * len(ctx.rules)
        return ms
    return t


def test_gains_are_kept_and_installed(monkeypatch):
    gains = {(LIN, 12, 2048, 4, 0): 1.0, (CYC, 14, 0, 0, 80): 0.5, (3, 1): 0.4}
    monkeypatch.setattr(autotune, "_time_batch", priced(gains))
    ctx = FakeCtx()
    res = autotune.autotune(ctx, batch(), context=64, reps=1)
    assert sorted(map(tuple, res["rules"])) == [(LIN, 12, 2048, 4, 0), (CYC, 14, 0, 0, 80)]
    assert res["launch"] == [3, 1]
    assert res["whole_batch_ms"]["kept"] and res["context_queries"] == 64
    assert res["whole_batch_ms"]["tuned"] == pytest.approx(10.0 - 1.9)
    assert sorted(ctx.rules) == sorted(map(tuple, res["rules"])) and ctx.launch == (3, 1)


def test_gains_below_the_margin_are_not_taken(monkeypatch):
    # 2 % of a 10 ms launch is below the 3 % margin
    gains = {(LIN, 12, 2048, 4, 0): 0.2, (2, 0): 0.2}
    monkeypatch.setattr(autotune, "_time_batch", priced(gains))
    ctx = FakeCtx()
    res = autotune.autotune(ctx, batch(), context=64, reps=1)
    assert res["rules"] == [] and res["launch"] == [0, 0]
    assert ctx.rules == [] and ctx.launch == (0, 0)


def test_result_dropped_when_the_whole_batch_is_slower(monkeypatch):
    """Gains inside the sample that turn into a loss on the whole batch: the
    library's rule stays."""
    gains = {(LIN, 12, 2048, 4, 0): 1.0, (CYC, 14, 0, 0, 80): 0.5}
    monkeypatch.setattr(autotune, "_time_batch", priced(gains, whole_penalty=1.0))
    ctx = FakeCtx()
    res = autotune.autotune(ctx, batch(), context=64, reps=1)
    assert not res["whole_batch_ms"]["kept"]
    assert res["whole_batch_ms"]["tuned"] > res["whole_batch_ms"]["library_rule"] * 0.97
    assert res["rules"] == [] and res["launch"] == [0, 0]
    assert ctx.rules == [] and ctx.launch == (0, 0)


def test_classes_are_tuned_largest_first(monkeypatch):
    seen = []

    def t(ctx, qs, reps):
        seen.append(tuple(ctx.rules[-1][:2]) if ctx.rules else None)
        return 10.0
    monkeypatch.setattr(autotune, "_time_batch", t)
    autotune.autotune(FakeCtx(), batch(), context=80, reps=1)
    order = [k for k in seen if k is not None]
    # the cyclic class holds 40 x (2^14 + 200) tuples, the linear one 40 x 3 x 2^12
    assert order.index((CYC, 14)) < order.index((LIN, 12))


def test_save_and_load_round_trip(tmp_path, monkeypatch):
    gains = {(LIN, 12, 4096, 2, 0): 1.0}
    monkeypatch.setattr(autotune, "_time_batch", priced(gains))
    res = autotune.autotune(FakeCtx(), batch(), context=64, reps=1)
    path = tmp_path / "tuning.json"
    autotune.save(res, str(path))
    back = autotune.load(str(path))
    assert back["rules"] == res["rules"] and back["launch"] == res["launch"]
    json.dumps(back)
    ctx = FakeCtx()
    autotune.install(ctx, back)
    assert ctx.rules == [tuple(r) for r in res["rules"]] and ctx.launch == tuple(res["launch"])
