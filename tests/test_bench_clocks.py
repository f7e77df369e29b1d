"""The benchmark's clock record (host logic, no GPU): the summary of the
nvidia-smi samples taken during the timed region, which decides whether a
run saw throttling.  Fed canned sample lines in nvidia-smi's
csv,noheader,nounits format (SM clock, max SM clock, then the hw_slowdown,
hw_thermal_slowdown, sw_thermal_slowdown and sw_power_cap reasons)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

IDLE = "Not Active, Not Active, Not Active, Not Active"


def _summary(lines):
    cs = bench.ClockSampler()
    cs.lines = lines
    return cs.summary()


def test_median_max_and_power_cap():
    s = _summary(["2070, 2070, " + IDLE,
                  "1980, 2070, Not Active, Not Active, Not Active, Active",
                  "2055, 2070, " + IDLE])
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_each_throttle_reason_is_reported():
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for i, name in enumerate(names):
        flags = ["Not Active"] * 4
        flags[i] = "Active"
        s = _summary(["1500, 2070, " + ", ".join(flags), "2070, 2070, " + IDLE])
        assert s["reasons"] == [name]


def test_malformed_and_unsupported_samples_are_skipped():
    s = _summary(["garbage", "[N/A], 2070, " + IDLE, "2070, 2070", "2000, 2070, " + IDLE])
    assert s["samples"] == 1 and s["sm_mhz"] == 2000.0


def test_no_samples_is_reported_as_unsampled():
    assert _summary([])["reasons"] == ["unsampled"]
    assert bench.ClockSampler().summary()["samples"] == 0  # never entered
