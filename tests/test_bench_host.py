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
    c.nvml = None  # the nvidia-smi path
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


class _FakeNvml:
    """Stands in for the NVML reader: replays (time, SM MHz, W, reason bits) samples."""
    max_mhz = 2070.0

    def __init__(self, rows):
        self.rows = list(rows)

    def sample(self):
        return self.rows.pop(0) if self.rows else None


def test_nvml_clock_summary_reasons_and_edges():
    c = bench.Clocks(0)
    c.nvml = _FakeNvml([(0.0, 2070.0, 300.0, 0x0)])
    c.edges = [c.nvml.sample()]
    c.samples = [(0.001, 2055.0, 1200.0, 0x1), (0.002, 2070.0, 1390.0, 0x4), (0.003, 2040.0, 1300.0, 0x0)]
    c.edges.append((0.004, 2070.0, 400.0, 0x0))
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["samples"] == 3 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # GPU-idle (0x1) is not a slowdown
    assert s["sm_mhz_before_after"] == [2070.0, 2070.0] and s["power_w_max"] == 1390.0
    c.samples.append((0.005, 1500.0, 700.0, 0x8 | 0x40))
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    # a region too short for the thread still reports the reads before and after it
    c.samples = []
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] == 2070.0


def test_traffic_only_for_the_same_kernel_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    entry = {"kernel_source_sha1": "abc", "dram_bytes_per_launch": 123}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"w/fp32/pull": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("abc", "w", "fp32", "pull") == 123
    assert bench._traffic("abd", "w", "fp32", "pull") is None  # counters of another source
    assert bench._traffic("abc", "w", "fp64", "pull") is None
    assert bench._traffic("abc", "other", "fp32", "pull") is None

