"""Host logic of bench.py that needs no GPU: the clock sampler that records
SM clocks and throttle reasons during the timed region (a fake nvidia-smi on
PATH plays the GPU), the roofline denominator read from the measured
peaks file, and the roofline arithmetic of the hop classes."""
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


def test_roofline_entries_arithmetic_and_captured_traffic():
    """The per-hop-class roofline entries: algorithmic bytes (8 links of 12
    reals and two spinors per site and rhs) over the mean launch time
    against the HBM peak for the inner hop, 1320 flop per site and rhs over
    the unit-count FP64 rate for the residual hop, and DRAM traffic only for
    a (precision, variant, rhs) combination with an ncu capture, scaled by
    the site count."""
    V = 48 * 48 * 48 * 96
    sites = V // 2
    prof = {"f16": {"launches": 10, "sites": 10.0 * sites, "site_rhs": 30.0 * sites, "ms": 10 * 1.0},
            "outer": {"launches": 4, "sites": 4.0 * sites, "site_rhs": 12.0 * sites, "ms": 4 * 23.6}}
    out = bench.roofline_entries(prof, "f16", "f64", V, 6766.0, "measured", 3, 106, 101)
    inner, outer = out["inner"], out["outer"]
    want_bytes = sites * (8 * 24 + 3 * 2 * 52)
    assert abs(inner["bytes_per_launch"] - want_bytes) < 1
    assert abs(inner["achieved"] - want_bytes / 1e-3 / 1e9) < 1e-6 * inner["achieved"]
    assert abs(inner["frac"] - inner["achieved"] / 6766.0) < 1e-12
    cap_sites, cap_bytes = bench.HOP_TRAFFIC[("f16", 106, 3)]
    assert abs(inner["traffic"] - cap_bytes * sites / cap_sites) < 1
    tf = 1320 * 3 * sites / 23.6e-3 / 1e12
    assert abs(outer["achieved"] - tf) < 1e-9 and abs(outer["frac"] - tf / bench.FP64_PEAK_TFLOPS) < 1e-12
    assert outer["traffic"] is not None and outer["fp64_pipe"]
    # a variant without a capture reports no traffic
    out = bench.roofline_entries(prof, "f16", "f64", V, 6766.0, "measured", 3, 101, 201)
    assert out["inner"]["traffic"] is None and out["outer"]["traffic"] is None
    # operands that fit in L2 get no HBM fraction
    small = {"f16": {"launches": 1, "sites": 1000.0, "site_rhs": 3000.0, "ms": 0.01},
             "outer": {"launches": 0, "sites": 0.0, "site_rhs": 0.0, "ms": 0.0}}
    out = bench.roofline_entries(small, "f16", "f64", 2000, 6766.0, "measured", 3, 106, 101)
    assert out["inner"]["frac"] is None and "outer" not in out
