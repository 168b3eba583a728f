"""Hop (dslash) kernel throughput versus lattice size, precision and number
of right-hand sides -- the GB300 counterpart of the paper's dslash
performance figure (Section 4).  Times wilson_hop-style launches of the
library's k_hop kernel on internal buffers with CUDA events (warm-up, then
back-to-back launches) and reports algorithmic GB/s (8 links per output
site, one input and one output spinor per site and rhs) and GFLOP/s at
1320 flop per output site and rhs.

python -m paper_1103_5103_gb300.dslash_bench [--dims 24x24x24x64 ...] [--prec f32 f16 f64] [--nrhs 1]
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import api, synth

LINK_B = {"f64": 144, "df": 144, "f32": 48, "f16": 24}  # FP64 and double-float links keep all three rows
SPINOR_B = {"f64": 192, "df": 192, "f32": 96, "f16": 52}


def run(dims, precs, nrhs=1, launches=50, eps=0.5, seed=2, rhs_block=1, variants=False, tune=False):
    lat = api.Lattice(dims)
    U = torch.from_numpy(synth.gauge_field(dims, eps, seed=seed)).cuda()
    g = api.Gauge(lat, U, precs=precs)
    del U
    Vh = lat.volume // 2
    psi = torch.from_numpy(synth.gaussian_source(dims, seed + 1)).cuda()
    rows = []
    for prec in precs:
        nb = lat.spinor_bytes(prec)
        stride = (nb + 255) // 256 * 256
        a = torch.empty(stride * nrhs, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        for r in range(nrhs):
            lat.spinor_import(psi, a[r * stride:(r + 1) * stride], prec, 1)
        if tune:
            rhs_block = -api.autotune(g, prec, nrhs)[0]
        choices = [-v for v in api.HOP_VARIANTS[prec]] if variants else [rhs_block]
        for rb in choices:
            for _ in range(5):
                api.hop_batch(g, a, b, nrhs, stride, 1.0, prec, 0, rb)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(launches):
                api.hop_batch(g, a, b, nrhs, stride, 1.0, prec, 0, rb)
            e1.record()
            torch.cuda.synchronize()
            s = e0.elapsed_time(e1) / launches / 1e3
            byts = Vh * 8 * LINK_B[prec] + Vh * nrhs * 2 * SPINOR_B[prec]
            rows.append({"dims": "x".join(map(str, dims)), "prec": prec, "nrhs": nrhs,
                         "variant" if rb < 0 else "rhs_block": -rb if rb < 0 else rb,
                         "us": s * 1e6, "GBps": byts / s / 1e9, "GFLOPs": 1320 * Vh * nrhs / s / 1e9})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", nargs="+", default=["8x8x8x8", "16x16x16x16", "16x16x16x32", "24x24x24x64",
                                                  "32x32x32x64"])
    ap.add_argument("--prec", nargs="+", default=["f64", "df", "f32", "f16"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--rhs-block", type=int, default=1)
    ap.add_argument("--launches", type=int, default=50)
    ap.add_argument("--variants", action="store_true", help="time every autotuner variant")
    ap.add_argument("--tune", action="store_true", help="time the variant the autotuner picks")
    args = ap.parse_args()
    for d in args.dims:
        dims = tuple(int(v) for v in d.split("x"))
        for row in run(dims, args.prec, args.nrhs, args.launches, rhs_block=args.rhs_block,
                       variants=args.variants, tune=args.tune):
            print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
