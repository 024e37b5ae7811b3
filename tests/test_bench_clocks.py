"""The benchmark's clock summary keeps the nvidia-smi samples taken inside the
timed region (host clock window) and reads their slowdown reasons."""
import datetime

import bench


def line(t, sm, reasons=()):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([ts, "0", str(sm), "2070", "700.5", "0x0"] + flags)


def test_samples_inside_the_window_win():
    t0 = 1_800_000_000.0
    lines = [line(t0 - 0.5, 1200), line(t0 + 0.002, 2040, ["sw_power_cap"]), line(t0 + 0.006, 2055),
             line(t0 + 0.3, 900, ["hw_slowdown"]), "garbage", ""]
    c = bench.summarize_clocks(lines, t0, t0 + 0.010)
    assert c["in_timed_region"] and c["samples"] == 2
    assert c["sm_mhz"] == (2040 + 2055) / 2 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]
    assert c["window_ms"] == 10.0


def test_no_sample_inside_falls_back_to_all():
    t0 = 1_800_000_000.0
    lines = [line(t0 - 0.2, 2070), line(t0 + 0.2, 2070, ["hw_thermal_slowdown"])]
    c = bench.summarize_clocks(lines, t0, t0 + 0.010)
    assert not c["in_timed_region"] and c["samples"] == 2
    assert c["reasons"] == ["hw_thermal_slowdown"]
    assert bench.summarize_clocks([], t0, t0 + 1) is None
