"""The benchmark's reference arm on the CPU: the oracle timed on the same
workload (a small graph here), reported in the line the benchmark's own arm
prints, with the reference-specific keys."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_has_the_contract_keys():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        warmup, steps, vertices = 1, 2, 1 << 11

    line = bench.run_reference(Args(), 0, 1)
    json.dumps(line)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # value is the step's input tuples over its mean time
    assert abs(line["value"] * line["ms_per_step"] * 1e-3 / line["config"]["tuples_per_step"] - 1) < 1e-9
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        warmup, steps, vertices = 0, 1, 1 << 10

    assert bench.run_reference(Args(), 1, 2) is None
