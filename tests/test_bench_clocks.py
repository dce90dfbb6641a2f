"""bench.py's clock record (the `clocks` key of the JSON line) from the
nvidia-smi samples taken during the timed region, on the CPU: median SM clock
of the bench's device, its maximum clock, and every throttle reason seen
active (the records that make a line rejected: hw_slowdown,
hw_thermal_slowdown, sw_thermal_slowdown; sw_power_cap is kept and noted)."""
import bench

ROWS = """\
0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
1, 1200, 2070, 300.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, [N/A], 2070, 1390.0, 0x0, Not Active, Not Active, Not Active, Not Active
0, 1965, 2070, 1400.1, 0x0000000000000008, Active, Not Active, Not Active, Not Active
garbage line
"""


def test_summary_of_device_zero(tmp_path):
    f = tmp_path / "clocks.csv"
    f.write_text(ROWS)
    s = bench.ClockSampler(str(f)).summary(0)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_other_device_and_missing_file(tmp_path):
    f = tmp_path / "clocks.csv"
    f.write_text(ROWS)
    s = bench.ClockSampler(str(f)).summary(1)
    assert s == {"sm_mhz": 1200.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 1}
    assert bench.ClockSampler(str(tmp_path / "none.csv")).summary(0) is None
    assert bench.ClockSampler(str(f)).summary(7) is None
