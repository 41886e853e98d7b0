"""Host logic of bench.py (no GPU): the clock record kept beside each number."""
import datetime

import bench

ROWS = """2026/12/04 04:32:22.900, 0, 1980, 2070, 610.2, 0x0, Not Active, Not Active, Not Active, Not Active
2026/12/04 04:32:23.000, 0, 2070, 2070, 905.1, 0x0, Not Active, Not Active, Not Active, Not Active
2026/12/04 04:32:23.100, 0, 2055, 2070, 1210.7, 0x4, Not Active, Not Active, Not Active, Active
2026/12/04 04:32:23.200, 0, 2070, 2070, 1190.0, 0x0, Not Active, Not Active, Not Active, Not Active
2026/12/04 04:32:23.300, 0, 1500, 2070, 400.0, 0x40, Not Active, Active, Not Active, Not Active
[N/A], 0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active
"""


def _t(s):
    return datetime.datetime.strptime("2026/12/04 04:32:" + s, "%Y/%m/%d %H:%M:%S.%f")


def test_parse_rows():
    rows = bench.ClockSampler.parse(ROWS)
    assert len(rows) == 5  # the row without a clock reading is dropped
    assert rows[0][0] == _t("22.900") and rows[0][1:3] == (1980.0, 2070.0)
    assert rows[2][3] == ["sw_power_cap"] and rows[4][3] == ["hw_thermal_slowdown"]


def test_summary_keeps_the_timed_region():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = _t("22.950"), _t("23.250")
    out = c.summarise(bench.ClockSampler.parse(ROWS))
    assert out["window"] == "timed region" and out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]  # the thermal row lies after the region


def test_summary_says_when_no_sample_is_inside():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = _t("23.310"), _t("23.390")
    out = c.summarise(bench.ClockSampler.parse(ROWS))
    assert out["window"].startswith("whole run") and out["samples"] == 5
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_unparsable_timestamps_fall_back_to_every_row():
    text = ROWS.replace("2026/12/04 04:32:23.100", "Thu Dec  4 04:32:23 2026")
    c = bench.ClockSampler(0)
    c.t0, c.t1 = _t("22.950"), _t("23.250")
    out = c.summarise(bench.ClockSampler.parse(text))
    assert out["samples"] == 2 and out["window"] == "timed region"
