"""Host-side pieces of bench.py that need no GPU: the clock record keeps only
the nvidia-smi samples taken inside the timed region and reports the
throttle reasons seen there."""
import datetime

import bench


def _line(t, sm, reason_cap="Not Active", reason_hw="Not Active"):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{ts}, 0, {sm}, 2070, 900.0, 0x0, {reason_hw}, Not Active, Not Active, {reason_cap}"


def test_clock_samples_outside_the_timed_region_are_ignored():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 1000.0, 1000.5
    c.lines = [_line(999.0, 345), _line(1000.1, 2070), _line(1000.3, 2055, reason_cap="Active"),
               _line(1001.5, 600, reason_hw="Active")]
    s = c.summary()
    assert s["samples"] == 2
    assert s["sm_mhz"] == (2070 + 2055) / 2 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]  # the idle sample's hw_slowdown is outside


def test_clock_summary_without_samples_in_the_region_says_so():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 1000.0, 1000.01
    c.lines = [_line(990.0, 2070)]
    s = c.summary()
    assert s["samples"] == 0 and "note" in s
