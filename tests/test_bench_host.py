"""Host logic of bench.py: the clock-sample summary that decides whether a run counts (throttle
reasons, median SM clock) and the lookup of a kernel's DRAM traffic, which must refuse counters
taken from another source of the kernel."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _clocks_from(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(line + "\n" for line in lines))
    c = bench.Clocks(0)
    c.path = str(p)
    c.proc = object()  # as if nvidia-smi had run
    return c.summary()


def test_clock_summary_median_and_reasons(tmp_path):
    na = "Not Active"
    rows = [f"0, {mhz}, 2070, 900.0, 0x0000000000000000, {na}, {na}, {na}, {na}" for mhz in (2070, 2055, 2070)]
    rows.append(f"0, 1980, 2070, 1400.0, 0x0000000000000004, {na}, {na}, {na}, Active")
    s = _clocks_from(tmp_path, rows)
    assert s["sm_mhz"] == 2062.5 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    rows.append(f"0, 1500, 2070, 700.0, 0x0000000000000008, Active, {na}, Active, {na}")
    s = _clocks_from(tmp_path, rows)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_ignores_malformed_lines(tmp_path):
    s = _clocks_from(tmp_path, ["garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
                                "0, 2070, 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 1 and s["reasons"] == []
    assert _clocks_from(tmp_path, ["garbage"]) is None


def test_traffic_only_for_the_same_kernel_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    entry = {"kernel_source_sha1": "abc", "dram_bytes_per_launch": 123}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"w/fp32/pull": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("abc", "w", "fp32", "pull") == 123
    assert bench._traffic("abd", "w", "fp32", "pull") is None  # counters of another source
    assert bench._traffic("abc", "w", "fp64", "pull") is None
    assert bench._traffic("abc", "other", "fp32", "pull") is None

