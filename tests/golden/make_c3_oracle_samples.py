"""Writes c3_oracle_samples.json: the FP64 oracle's solution of the 24^3x64
benchmark workload (eps 0.5, gauge seed 3, point source at site 0, spin 0,
colour 0) for the heaviest and the lightest mass, at the source site, its
eight neighbours and 128 random sites.

The solutions come from the oracle's even-odd BiCGstab (Section 6.2.3, Eq.
eo2-eo4) run to a 1e-13 relative residual, so they are exact to well below
the 1e-8 the GPU solutions are compared at.  Only oracle/ and the shared
input generator are used.  It takes a few minutes on one core:

    python tests/golden/make_c3_oracle_samples.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1103_5103_gb300 import synth  # noqa: E402

DIMS = (24, 24, 24, 64)
EPS, SEED = 0.5, 3
MASSES = [0.40, 0.05]


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


def main():
    U = synth.gauge_field(DIMS, EPS, seed=SEED)
    b = synth.point_source(DIMS, 0, 0)
    sites = sample_sites(DIMS)
    out = {"what": "FP64 oracle even-odd BiCGstab solutions of M_k(m0) x = b (kappa form) at sampled sites",
           "dims": list(DIMS), "eps": EPS, "gauge_seed": SEED, "source": {"site": 0, "spin": 0, "colour": 0},
           "tol": 1e-13, "sites": sites, "masses": MASSES, "x": {}, "true_relres": {}, "iterations": {}}
    for m in MASSES:
        x, st = O.eo_solve(U, DIMS, b, m, tol=1e-13)
        xs = x[sites].reshape(len(sites), 12)
        out["x"][repr(m)] = [[[float(v.real), float(v.imag)] for v in row] for row in xs]
        out["true_relres"][repr(m)] = st["true_relres_full"]
        out["iterations"][repr(m)] = st["iterations"]
        print(m, st, flush=True)
    with open(os.path.join(HERE, "c3_oracle_samples.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
