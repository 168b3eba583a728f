"""Run by tests/test_checked_build_gpu.py in a process of its own with
WL_LIBRARY=checked: a pass over the library's kernels -- every operator in
every precision on the tiny and odd lattices, every hop variant with a
ragged rhs group, the solvers in each mode and precision pair, the
multi-shift solver, the backward and the no-allocation dslash -- in the
bounds-checked build, then the recorded violations (none expected).
Prints one JSON line."""
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1103_5103_gb300 import api, synth  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def main():
    assert api.is_checked_build()
    calls = 0
    for dims in [(2, 2, 2, 2), (6, 4, 4, 8), (4, 6, 2, 10), (8, 4, 4, 8)]:
        lat = api.Lattice(dims)
        g = api.Gauge(lat, cuda(synth.gauge_field(dims, 0.5, seed=3)))
        psi = cuda(synth.gaussian_source(dims, seed=4))
        out = torch.empty_like(psi)
        for prec in ("f64", "f32", "f16", "df"):
            for op in (api.OP_HOP, api.OP_M, api.OP_MPREC):
                api.wilson_dslash(g, psi, out, 0.12, prec, op)
                api.wilson_dslash_dag(g, psi, out, 0.12, prec, op)
                api.wilson_dslash_noalloc(g, psi, out, 0.12, prec, op)
                calls += 3
            stride = (lat.spinor_bytes(prec) + 255) // 256 * 256
            nrhs = 5
            a = torch.zeros(stride * nrhs, dtype=torch.uint8, device="cuda")
            for r in range(nrhs):
                lat.spinor_import(psi, a[r * stride:(r + 1) * stride], prec, 0)
            for v in api.HOP_VARIANTS[prec]:
                b = torch.zeros_like(a)
                try:
                    api.hop_batch(g, a, b, nrhs, stride, 1.0, prec, 1, -v)
                    calls += 1
                except api.WilsonError as e:
                    # TMA tiles need X/2 a multiple of 4
                    assert v >= 9000 and e.status == api.WL_ERR_ARG, (dims, prec, v, e)
        bs = [cuda(synth.point_source(dims, 1, 2)), cuda(synth.z2_source(dims, 5))]
        masses = [0.4, 0.1]
        for inner, outer, mode in (("f32", "f64", api.MODE_GRAPH), ("f16", "f64", api.MODE_HOST),
                                   ("f64", "f64", api.MODE_GRAPH), ("f32", "df", api.MODE_PERSISTENT),
                                   ("f16", "df", api.MODE_GRAPH)):
            api.multimass_solve(g, bs, masses, api.params(inner_prec=inner, outer_prec=outer, mode=mode,
                                                          guess=api.GUESS_SSM if inner == "f16" else api.GUESS_POLY))
            calls += 1
        api.multimass_solve(g, bs, masses, api.params(inner_prec="f16", outer_blocks_per_sm=1, verify_full=1))
        rh = cuda(synth.gaussian_source(dims, seed=6))
        for outer in ("f64", "df"):
            xs = [torch.empty_like(psi) for _ in masses]
            api.bicgstab_m_solve(g, bs[0], xs, masses, api.params(outer_prec=outer, shadow=rh))
            calls += 1
        g.close()
    dims = (4, 4, 4, 4)
    lat = api.Lattice(dims)
    U = cuda(synth.gauge_field(dims, 0.3, seed=7))
    g = api.Gauge(lat, U, precs=("f64", "f32", "df"))
    b = cuda(synth.gaussian_source(dims, seed=8))
    masses = [0.3, 0.1]
    xs, _ = api.multimass_solve(g, [b], masses, api.params())
    api.solve_backward(g, b, [2 * xs[0][i] for i in range(2)], masses, xs=[xs[0][i] for i in range(2)])
    api.solve_backward(g, b, [2 * xs[0][i] for i in range(2)], masses)   # re-solve
    calls += 2
    first = api.checked_status()
    print(json.dumps({"checked_build": True, "calls": calls, "first_violation": first}))
    return 0 if first == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
