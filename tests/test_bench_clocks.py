"""The benchmark's clock record: nvidia-smi samples taken during the timed region are reduced to the
median SM clock under load, the maximum clock and the throttle reasons seen active.  A stand-in
nvidia-smi on PATH prints fixed samples, so this runs without a GPU."""
import os
import stat
import sys
import time

from conftest import ROOT

SAMPLES = """0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1995, 2070, 1398.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 2070, 2070, 1120.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, [N/A], 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 2055, 2070
0, 1980, 2070, 1400.0, 0x0000000000000020, Not Active, Not Active, Active, Not Active
"""


def _fake_smi(tmp_path, text):
    data = tmp_path / "samples.txt"
    data.write_text(text)
    exe = tmp_path / "nvidia-smi"
    exe.write_text(f"#!/bin/sh\ncat '{data}'\nexec sleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_clock_record_median_max_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, SAMPLES) + os.pathsep + os.environ.get("PATH", ""))
    sys.path.insert(0, ROOT)
    import bench

    c = bench.Clocks(0)
    time.sleep(0.5)   # the stand-in has printed its samples by now
    rec = c.stop()
    # four well-formed samples (a clock of [N/A] and a short line are skipped)
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == (1995 + 2070) / 2 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory: no nvidia-smi to start
    sys.path.insert(0, ROOT)
    import bench

    rec = bench.Clocks(0).stop()
    assert rec["sm_mhz"] is None and rec["sm_max_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
