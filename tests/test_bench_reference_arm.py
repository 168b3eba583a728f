"""The reference arm of bench.py (`--impl reference`) times the FP64 oracle
on the host. These CPU tests pin the JSON line it prints: the keys the
benchmark contract needs, the scaling of the sampled time per BiCGstab
iteration by the step's iteration count, rank 0 alone printing, and the
`unavailable` line for a workload without a recorded iteration count."""
import argparse
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(config="c3", steps=2, warmup=3):
    return argparse.Namespace(config=config, steps=steps, warmup=warmup, gpus=1)


def _tiny_cfg():
    cfg = dict(bench.CONFIGS["c3"])
    cfg["dims"] = (4, 4, 4, 4)   # the line's composition does not depend on the lattice
    return cfg


def test_reference_line_keys_and_scaling(monkeypatch, capsys):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    per_iter = [0.5, 0.5, 0.5, 2.0, 4.0]   # warm-up samples first, then the timed ones
    calls = []

    def fake_sample(cfg, U, bs, target_s=15.0):
        calls.append(target_s)
        return per_iter[len(calls) - 1], 3, 1.0

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    bench.run_reference(_args(), _tiny_cfg())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    n = bench.REF_ITERS_PER_STEP["c3"]
    assert len(calls) == 5                      # 3 warm-up + 2 timed samples
    assert line["impl"] == "reference"
    assert line["value"] == pytest.approx(n * (2.0 + 4.0) / 2)   # mean of the timed steps only
    assert line["ms_per_step"] == pytest.approx(line["value"] * 1e3)
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["higher_is_better"] is False and line["steps"] == 2 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.CONFIGS["c3"]["name"]
    # each sample is bounded so that the whole run takes about 90 s
    assert all(5.0 <= t <= 90.0 for t in calls)


def test_reference_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: pytest.fail("rank 1 ran the oracle"))
    bench.run_reference(_args(), _tiny_cfg())
    assert capsys.readouterr().out == ""


def test_reference_without_iteration_count_is_unavailable():
    """The 16^3x32 workload has no recorded step iteration count: the arm
    prints its unavailable line and exits 0 (run as the driver runs it)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unavailable"]
