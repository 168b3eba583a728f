"""Writes <config>_oracle_multimass.json: the FP64 oracle's run of the paper's
single-mass multi-mass scheme (Section 6.2, Section 7: masses heaviest
first, Lagrange guess through all earlier solutions, even-odd BiCGstab to a
1e-10 residual) on a benchmark workload, per point source and mass:

  iterations  -- the oracle's BiCGstab iterations at tol 1e-10 (the count
                 the benchmark's oracle arm scales its timed iteration by);
  x           -- the solution polished by the oracle's even-odd BiCGstab to
                 a 1e-13 residual (exact to far below the 1e-8 the GPU
                 solutions are compared at), at the source site, its eight
                 neighbours and random sites (128 drawn, 32 kept).

Only oracle/ and the shared input generator are used.  The oracle's
per-site loops run on all host cores (OMP_NUM_THREADS to change):

    python tests/golden/make_oracle_multimass.py --config c3 --sources 0 1 ... 11 --trim 32
    python tests/golden/make_oracle_multimass.py --config c5 --sources 0 11 --trim 32

24^3x64 takes a few minutes per source on eight cores, 48^3x96 about an
hour and 50 GB of host memory.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1103_5103_gb300 import synth  # noqa: E402

WORKLOADS = {
    "c3": dict(dims=(24, 24, 24, 64), eps=0.5, seed=3, masses=[0.40, 0.35, 0.30, 0.25, 0.20, 0.15, 0.10, 0.05]),
    "c5": dict(dims=(48, 48, 48, 96), eps=0.7, seed=5, masses=[0.5 * 0.04 ** (i / 15.0) for i in range(16)]),
}
TOL, POLISH_TOL = 1e-10, 1e-13


def sample_sites(dims, n_random=128, seed=7):
    X, Y, Z, T = dims
    V = X * Y * Z * T
    nb = [0]
    for mu, ext in enumerate(dims):
        for d in (1, -1):
            c = [0, 0, 0, 0]
            c[mu] = d % ext
            nb.append(c[0] + X * (c[1] + Y * (c[2] + Z * c[3])))
    rng = np.random.default_rng(seed)
    return sorted(set(nb) | set(int(v) for v in rng.choice(V, size=n_random, replace=False)))


def trim(path, n_random):
    """Keep the source site, its neighbours and the n_random lowest of the
    stored random sites (the file stays a few hundred kB to a few MB)."""
    with open(path) as f:
        out = json.load(f)
    dims = out["dims"]
    keep_nb = set(sample_sites(dims, n_random=0))
    sites = out["sites"]
    rand = sorted(s for s in sites if s not in keep_nb)[:n_random]
    keep = sorted(keep_nb | set(rand))
    idx = [sites.index(s) for s in keep]
    for rec in out["sources"].values():
        rec["x"] = [None if x is None else [x[i] for i in idx] for x in rec["x"]]
    out["sites"] = keep
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", choices=sorted(WORKLOADS), required=True)
    ap.add_argument("--sources", type=int, nargs="*", default=[0],
                    help="spin-colour point sources k = 3 * spin + colour")
    ap.add_argument("--trim", type=int, default=0,
                    help="afterwards keep only the source neighbourhood and this many random sites")
    args = ap.parse_args()
    w = WORKLOADS[args.config]
    dims, masses = w["dims"], w["masses"]
    path = os.path.join(HERE, f"{args.config}_oracle_multimass.json")
    if not args.sources and args.trim:
        trim(path, args.trim)
        return
    out = json.load(open(path)) if os.path.exists(path) else {
        "what": "FP64 oracle multi-mass scheme (Lagrange guess, even-odd BiCGstab) per point source and mass: "
                "iterations at tol 1e-10 and the solution polished to 1e-13 at sampled sites",
        "dims": list(dims), "eps": w["eps"], "gauge_seed": w["seed"], "masses": masses, "tol": TOL,
        "polish_tol": POLISH_TOL, "sites": sample_sites(dims), "sources": {}}
    sites = out["sites"]
    threads = O.set_threads()
    U = synth.gauge_field(dims, w["eps"], seed=w["seed"])
    for k in args.sources:
        b = synth.point_source(dims, k // 3, k % 3)
        rec = {"iterations": [None] * len(masses), "restarts": [None] * len(masses),
               "true_relres": [None] * len(masses), "polish_iterations": [None] * len(masses),
               "x": [None] * len(masses)}
        t0 = time.time()

        def on_solution(i, x, st):
            m = masses[i]
            xe = x.copy()
            xe[O.parity_mask(dims)] = 0
            xp, sp = O.eo_solve(U, dims, b, m, x0e=xe, tol=POLISH_TOL)
            del xe
            rec["iterations"][i] = st["iterations"]
            rec["restarts"][i] = st["restarts"]
            rec["true_relres"][i] = st["true_relres_full"]
            rec["polish_iterations"][i] = sp["iterations"]
            rec["x"][i] = [[[float(v.real), float(v.imag)] for v in row]
                           for row in xp[sites].reshape(len(sites), 12)]
            print(f"source {k} m0 {m:.5f}: {st['iterations']} iterations, true relres "
                  f"{st['true_relres_full']:.2e}; polish {sp['iterations']} -> {sp['true_relres_full']:.2e} "
                  f"({time.time() - t0:.0f} s)", flush=True)

        O.multimass_solve(U, dims, b, masses, tol=TOL, on_solution=on_solution)
        rec["seconds"] = time.time() - t0
        rec["threads"] = threads
        out["sources"][str(k)] = rec
        with open(path, "w") as f:
            json.dump(out, f, separators=(",", ":"))
    if args.trim:
        trim(path, args.trim)


if __name__ == "__main__":
    main()
