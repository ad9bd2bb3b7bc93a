"""bench.py's clock record, from a fake nvidia-smi log: only the samples
stamped inside the timed region count, throttle reasons are read from their
columns, and a log without usable stamps falls back to every sample."""
import datetime
import subprocess
import tempfile
from unittest import mock

import bench


def _stamp(t):
    return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


def _clocks(lines, t0):
    c = bench.Clocks.__new__(bench.Clocks)
    c.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.f.write("\n".join(lines) + "\n")
    c.f.flush()
    c.p = subprocess.Popen(["sleep", "30"])
    c.t0 = t0
    return c


def test_samples_inside_the_timed_region_only():
    t0 = 1.0e9
    na = "Not Active"
    lines = [f"{_stamp(t0 - 1.0)}, 0, 1200, 2032, 200.0, 0x0, Active, {na}, {na}, {na}",  # before: hw_slowdown
             f"{_stamp(t0 + 0.05)}, 0, 2032, 2032, 900.0, 0x4, {na}, {na}, {na}, Active",
             f"{_stamp(t0 + 0.15)}, 0, 2020, 2032, 950.0, 0x0, {na}, {na}, {na}, {na}",
             f"{_stamp(t0 + 5.0)}, 0, 1000, 2032, 100.0, 0x0, {na}, {na}, Active, {na}"]  # after
    c = _clocks(lines, t0)
    with mock.patch("time.time", return_value=t0 + 0.2):
        rec = c.stop()
    assert rec == {"sm_mhz": 2026.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 2,
                   "samples_in_timed_region": 2}


def test_unstamped_log_keeps_every_sample():
    na = "Not Active"
    lines = [f"bad-stamp, 0, 2032, 2032, 900.0, 0x0, {na}, {na}, {na}, {na}",
             f"bad-stamp, 0, 1800, 2032, 900.0, 0x0, {na}, Active, {na}, {na}"]
    c = _clocks(lines, 1.0e9)
    rec = c.stop()
    assert rec["samples"] == 2 and rec["samples_in_timed_region"] == 0
    assert rec["sm_mhz"] == 1916.0 and rec["reasons"] == ["hw_thermal_slowdown"]
