"""Host-side logic of bench.py that needs no GPU: the clock-sample parser
that decides which throttle reasons a run reports (CPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# `nvidia-smi --query-gpu=<bench.Clocks.FIELDS> --format=csv,noheader,nounits` lines
IDLE = "0, 2070, 2070, 212.31, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAPPED = "0, 1965, 2070, 1398.90, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
THERMAL = "0, 1800, 2070, 1250.00, 0x0000000000000020, Not Active, Not Active, Active, Not Active"
HW = "0, 1500, 2070, 900.00, 0x0000000000000008, Active, Active, Not Active, Not Active"


def test_clean_run():
    out = bench.parse_clocks([IDLE, IDLE, IDLE])
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": []}


def test_reasons_are_collected_and_the_clock_is_the_median():
    out = bench.parse_clocks([IDLE, CAPPED, THERMAL, HW, IDLE])
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1965.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 5
    assert bench.parse_clocks([IDLE, CAPPED])["reasons"] == ["sw_power_cap"]


def test_unusable_lines_are_skipped():
    assert bench.parse_clocks([]) is None
    assert bench.parse_clocks(["", "garbage", "0, [N/A], [N/A], [N/A], 0x0, Not Active, Not Active, "
                                              "Not Active, Not Active"]) is None
    out = bench.parse_clocks(["0, 2070", IDLE + "\n"])
    assert out["samples"] == 1 and out["reasons"] == []


def test_query_fields_match_the_parser():
    fields = bench.Clocks.FIELDS.split(",")
    assert len(fields) == 9 and fields[1] == "clocks.sm" and fields[2] == "clocks.max.sm"
    assert [f.split(".")[-1] for f in fields[5:9]] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                                      "sw_power_cap"]
