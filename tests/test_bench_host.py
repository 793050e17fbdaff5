"""Host logic of bench.py that needs no GPU: parsing of the nvidia-smi clock
samples taken during the timed region (a run that saw a hardware or thermal
slowdown must be recognisable), and the key of the DRAM-traffic record."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_rows_median_max_and_reasons():
    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2050, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1500, 2070, 700.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.parse_clock_rows(text)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2050.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_rows_empty():
    c = bench.parse_clock_rows("")
    assert c == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_record_keyed_to_the_search_kernel_sources():
    # the key is a hash of the files the kernel is built from: stable across calls
    assert bench._src_sha() == bench._src_sha()
    assert len(bench._src_sha()) == 16
    assert set(bench.ICP_TRAFFIC) == {"bytes", "src_sha"}


def test_clock_rejection_rule():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 10}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected({**ok, "sm_mhz": 1800.0, "reasons": ["sw_power_cap"]})
    assert bench.clocks_rejected({**ok, "reasons": ["hw_slowdown"]})
    assert bench.clocks_rejected({**ok, "reasons": ["sw_thermal_slowdown", "sw_power_cap"]})
    assert bench.clocks_rejected({**ok, "sm_mhz": 1400.0})  # stuck low, no reason
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                      "reasons": ["unavailable"], "samples": 0})
