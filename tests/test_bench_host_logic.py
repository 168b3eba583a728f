"""Host logic of bench.py that needs no GPU: the clock sampler that records
SM clocks and throttle reasons during the timed region (a fake nvidia-smi on
PATH plays the GPU), and the roofline denominator read from the measured
peaks file."""
import json
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# index, clocks.sm, clocks.max.sm, power.draw, active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
ROWS = [
    "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1100.2, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    "0, [N/A], 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
]


def _fake_smi(tmp_path, rows):
    """An executable named nvidia-smi that prints the rows once and then
    waits, as `nvidia-smi -lms` does until it is terminated."""
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{r}'" for r in rows)
    script.write_text(f"#!/bin/sh\n{body}\nexec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_median_max_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, ROWS) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    time.sleep(1.0)
    c = s.stop()
    assert c["samples"] == 4
    assert c["sm_mhz"] == 2070.0            # median of 2070, 1980, 2070 (the N/A row has no clock)
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory: no nvidia-smi
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6689.8, "bf16_tflops": 1900.0}))
    assert bench.measured_peaks() == (6689.8, "measured")
