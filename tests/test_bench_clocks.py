"""The clock record of the bench line (no GPU): nvidia-smi samples taken during the timed
region are summarised as the median SM clock under load, the maximum clock, the largest
power draw and every throttle reason that was active in any sample."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sampler_with(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(l + "\n" for l in lines))
    c = bench.ClockSampler(0)
    c.proc, c.path = object(), str(path)  # as if nvidia-smi had written the file
    return c


def row(mhz, power, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return f"0, {mhz}, 2070, {power}, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}"


def test_median_under_load_and_no_reason(tmp_path):
    lines = [row(1965, 120.0), row(2070, 480.0), row(2055, 510.5), row(2070, 530.0)]
    s = sampler_with(tmp_path, lines).summary()
    assert s["sm_mhz"] == 2070.0  # median of the three samples above 200 W
    assert s["sm_max_mhz"] == 2070.0 and s["power_w_max"] == 530.0
    assert s["samples"] == 4 and s["reasons"] == []


def test_every_active_reason_is_reported(tmp_path):
    lines = [row(2070, 600.0, cap="Active"), row(1800, 610.0, hw_th="Active"),
             row(2070, 590.0, hw="Active", sw_th="Active")]
    s = sampler_with(tmp_path, lines).summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_idle_samples_only_and_malformed_lines(tmp_path):
    lines = ["", "garbage", "0, [N/A], 2070, 90.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             row(1200, 95.0), row(1300, 99.0)]
    s = sampler_with(tmp_path, lines).summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 1250.0  # no sample under load: median of all


def test_no_samples_and_no_sampler(tmp_path):
    assert sampler_with(tmp_path, []).summary()["reasons"] == ["no samples"]
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]
