"""Initial-guess gain per mass, the experiment of Section 7 that compares
polynomial extrapolation of growing order with solution-space minimisation.

Runs multimass_solve on one synthetic workload with the zero guess, with the
Lagrange guess through the last n = 1 .. N-1 solutions, and with the
solution-space minimisation guess through the last n solutions, and prints
one JSON line per setting: inner iterations, outer restarts and seconds per
mass, the step time, and the paper's gain = total iterations with the guess
divided by total iterations with the zero guess (below 1 is better), also
per mass.

python -m paper_1103_5103_gb300.guess_gain [--dims 16x16x16x32] [--eps 0.5]
       [--sources z2|points12] [--inner f32] [--repeat 2]
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import api, synth

MASSES = [0.40, 0.35, 0.30, 0.25, 0.20, 0.15, 0.10, 0.05]


def sources(dims, kind, seed):
    if kind == "points12":
        return [synth.point_source(dims, s, c) for s in range(4) for c in range(3)]
    return [synth.z2_source(dims, seed=seed)]


def run(dims, eps, seed, kind, inner, repeat, masses=MASSES):
    lat = api.Lattice(dims)
    g = api.Gauge(lat, torch.from_numpy(synth.gauge_field(dims, eps, seed=seed)).cuda())
    bs = [torch.from_numpy(b).cuda() for b in sources(dims, kind, seed + 1)]
    xs = [[torch.empty_like(b) for _ in masses] for b in bs]
    settings = [("zero", 0)] + [("poly", n) for n in range(1, len(masses))] + \
               [("ssm", n) for n in range(1, len(masses))]
    code = {"zero": api.GUESS_ZERO, "poly": api.GUESS_POLY, "ssm": api.GUESS_SSM}
    base = None
    rows = []
    for guess, n in settings:
        prm = api.params(guess=code[guess], guess_max=n, inner_prec=inner)
        for _ in range(repeat):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = api.multimass_solve(g, bs, masses, prm, xs=xs)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        its = [sum(st[r][i]["iterations"] for r in range(len(bs))) for i in range(len(masses))]
        row = {"dims": "x".join(map(str, dims)), "eps": eps, "sources": kind, "inner": inner, "guess": guess,
               "order": n, "masses": masses, "iterations_per_mass": its,
               "restarts_per_mass": [sum(st[r][i]["restarts"] for r in range(len(bs))) for i in range(len(masses))],
               "seconds_per_mass": [st[0][i]["seconds"] for i in range(len(masses))],
               "max_true_relres": max(s["true_relres"] for row_ in st for s in row_), "step_s": dt}
        if base is None:
            base = its
        row["gain"] = sum(its) / max(1, sum(base))
        row["gain_per_mass"] = [i_ / max(1, b_) for b_, i_ in zip(base, its)]
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="16x16x16x32")
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--sources", choices=["z2", "points12"], default="z2")
    ap.add_argument("--inner", choices=["f64", "f32", "f16"], default="f32")
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()
    run(tuple(int(v) for v in args.dims.split("x")), args.eps, args.seed, args.sources, args.inner, args.repeat)


if __name__ == "__main__":
    main()
