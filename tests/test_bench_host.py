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


def test_traffic_records_keyed_to_each_kernels_sources(monkeypatch):
    # the key is a hash of the files the kernel is built from: stable across
    # calls, different per kernel; a record is reported only while it matches
    for k in bench.TRAFFIC:
        assert bench.src_sha(k) == bench.src_sha(k) and len(bench.src_sha(k)) == 16
        assert set(bench.TRAFFIC[k]) == {"bytes", "src_sha"}
    assert len({bench.src_sha(k) for k in bench.TRAFFIC}) == len(bench.TRAFFIC)
    monkeypatch.setitem(bench.TRAFFIC, "k_knn", {"bytes": 123, "src_sha": bench.src_sha("k_knn")})
    assert bench.traffic_of("k_knn") == 123
    monkeypatch.setitem(bench.TRAFFIC, "k_knn", {"bytes": 123, "src_sha": "0" * 16})
    assert bench.traffic_of("k_knn") is None


def test_summary_keeps_listed_keys_in_order():
    rec = {"a": 1.23456789, "b": 2, "c": "x"}
    assert bench._summary(rec, ("c", "a", "missing")) == {"c": "x", "a": 1.23457}
    assert bench._summary(None, ("a",)) is None
    assert bench._sig(7.756328758e-08) == 7.756e-08 and bench._sig(12983.3246) == 12980.0
    assert bench._sig(0.0) == 0.0 and bench._sig(3) == 3


def test_clock_rejection_rule():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 10}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected({**ok, "sm_mhz": 1800.0, "reasons": ["sw_power_cap"]})
    assert bench.clocks_rejected({**ok, "reasons": ["hw_slowdown"]})
    assert bench.clocks_rejected({**ok, "reasons": ["sw_thermal_slowdown", "sw_power_cap"]})
    assert bench.clocks_rejected({**ok, "sm_mhz": 1400.0})  # stuck low, no reason
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                      "reasons": ["unavailable"], "samples": 0})
