"""Host-side pieces of bench.py that decide whether a number is kept: the clock
record taken from nvidia-smi during the timed region, and the traffic figure's
tie to the kernel sources. Run without a GPU (nvidia-smi is a stand-in script)."""
import os
import stat
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_smi(tmp_path, lines):
    p = tmp_path / "nvidia-smi"
    body = "".join(f"echo '{ln}'\n" for ln in lines)
    p.write_text("#!/bin/sh\n" + body + "exec sleep 30\n")
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def _sample(tmp_path, monkeypatch, lines):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    import time
    time.sleep(0.5)
    return s.stop()


def test_clock_record_under_load(tmp_path, monkeypatch):
    idle = "1200, 2070, 0x0, Not Active, Not Active, Not Active, Not Active, 0"
    busy = "2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active, 100"
    capped = "1965, 2070, 0x4, Not Active, Not Active, Not Active, Active, 100"
    r = _sample(tmp_path, monkeypatch, [idle, busy, busy, capped])
    # idle samples are left out; the median is over the three loaded ones
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_reports_thermal_slowdown(tmp_path, monkeypatch):
    hot = "1500, 2070, 0x20, Not Active, Not Active, Active, Not Active, 99"
    r = _sample(tmp_path, monkeypatch, [hot, hot])
    assert r["reasons"] == ["sw_thermal_slowdown"] and r["sm_mhz"] == 1500.0


def test_traffic_is_null_once_the_kernel_sources_change(monkeypatch):
    import json
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        stored = json.load(f)["radix_scatter"]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: stored["source_digest"])
    assert bench.ncu_traffic("radix_scatter") == stored["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0000000000000000")
    assert bench.ncu_traffic("radix_scatter") is None
