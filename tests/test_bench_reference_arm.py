"""The reference arm of bench.py (`--impl reference`) times the FP64 oracle
on the host. These CPU tests pin the JSON line it prints: the keys the
benchmark contract needs, the scaling of the sampled oracle times by the
oracle's own iteration counts (stored by an oracle-only script under
tests/golden, never taken from the optimised arm), rank 0 alone printing,
and the `unavailable` line for a workload without stored counts."""
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


COUNTS = {"iterations": [10.0, 8.0, 3.0], "restarts": [2.0, 1.0, 0.0], "sources": [0, 11],
          "file": "tests/golden/c3_oracle_multimass.json"}


def test_reference_line_keys_and_scaling(monkeypatch, capsys):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    # the calibration (M_prec 1.0 s, iteration 2.5 s), then per step one
    # application: warm-up first, then the timed ones
    samples = [(1.0, 2.5, 9.0)] + [(1.0, None, 1.0)] * 3 + [(1.0, None, 1.0), (2.0, None, 2.0)]
    calls = []

    def fake_sample(cfg, U, b, iteration=True):
        calls.append(iteration)
        assert iteration == (len(calls) == 1)
        return samples[len(calls) - 1]

    monkeypatch.setattr(bench, "oracle_sample", fake_sample)
    monkeypatch.setattr(bench, "oracle_counts", lambda config: COUNTS)
    monkeypatch.setattr(bench, "oracle_threads", lambda: 4)
    bench.run_reference(_args(), _tiny_cfg())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 6                      # calibration, 3 warm-up + 2 timed samples

    def step(t_mprec, t_iter):   # 12 sources; per mass iterations x t_iter + (4.5 + restarts) x t_mprec
        return 12 * sum(i * t_iter + (4.5 + r) * t_mprec for i, r in zip(COUNTS["iterations"], COUNTS["restarts"]))
    assert line["impl"] == "reference"
    assert line["value"] == pytest.approx((step(1.0, 2.5) + step(2.0, 5.0)) / 2)   # timed steps only
    assert line["ms_per_step"] == pytest.approx(line["value"] * 1e3)
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["higher_is_better"] is False and line["steps"] == 2 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 4
    assert line["cpu_baseline"]["value"] == line["value"]
    sample = line["cpu_baseline"]["sample"]
    assert "oracle's own 252 iterations" in sample and COUNTS["file"] in sample
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.CONFIGS["c3"]["name"]


def test_oracle_counts_come_from_the_oracle_only_golden_file():
    """The counts the reference arm scales by are the oracle's own, stored
    by tests/golden/make_oracle_multimass.py (which imports only oracle/ and
    the input generator) for the 24^3x64 and 48^3x96 workloads."""
    src = open(os.path.join(ROOT, "tests", "golden", "make_oracle_multimass.py")).read()
    assert "from oracle import oracle" in src and "api" not in src.replace("argparse", "")
    for config, n_mass in (("c3", 8), ("c5", 16)):
        c = bench.oracle_counts(config)
        if c is None:
            pytest.skip(f"no stored oracle counts for {config}")
        assert len(c["iterations"]) == n_mass and all(v > 0 for v in c["iterations"])
        assert len(c["restarts"]) == n_mass and c["sources"]


def test_reference_other_ranks_print_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: pytest.fail("rank 1 ran the oracle"))
    bench.run_reference(_args(), _tiny_cfg())
    assert capsys.readouterr().out == ""


def test_reference_without_iteration_count_is_unavailable():
    """The 16^3x32 workload has no recorded step iteration count: the arm
    prints its unavailable line and exits 0 (run as a separate process,
    the way the command line launches it)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unavailable"]
