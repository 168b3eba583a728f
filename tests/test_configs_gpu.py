"""The benchmark workloads at their full sizes, in the launch configuration
the benchmark times, checked against the FP64 oracle per mass, with the
outer loop in FP64 (the paper's double precision, the benchmark's setting)
and in double-float.

16^3x32 and 24^3x64: the oracle's full-lattice true residual ||b - M_k x|| /
||b|| of every GPU solution it can afford (one oracle matvec each); on
24^3x64 also every solution against the oracle's own multi-mass run,
polished to 1e-13, stored at sampled sites for all twelve sources and eight
masses (tests/golden/c3_oracle_multimass.json).
48^3x96: the oracle residual at 4096 random sites plus the source site and
its neighbours (one oracle matvec takes seconds there), and the solutions
of the sources the oracle could afford against its stored solutions
(tests/golden/c5_oracle_multimass.json).  Every mass must reach the 1e-10
true residual the solver promises, and every solution must agree with the
oracle's to 1e-8."""
import json
import os

import numpy as np
import pytest
import torch

from helpers import SampledResidual, rel
from oracle import oracle as O
from paper_1103_5103_gb300 import synth

pytestmark = pytest.mark.gpu

MASSES8 = [0.40, 0.35, 0.30, 0.25, 0.20, 0.15, 0.10, 0.05]
MASSES16 = [0.5 * 0.04 ** (i / 15.0) for i in range(16)]
TOL = 1e-10
# the oracle recomputes the residual in its own rounding order
SLACK = 1.02


@pytest.fixture(scope="module")
def api():
    from paper_1103_5103_gb300 import api
    return api


@pytest.fixture(autouse=True)
def _release_cached_memory():
    yield
    import gc
    gc.collect()
    torch.cuda.empty_cache()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_16c32_z2_source_all_masses(api, inner):
    """16^3x32, eps 0.5, one Z2 source, 8 masses: every mass at a 1e-10 oracle
    true residual; the BiCGstab-M solutions (FP64 vectors alongside the FP32
    inner case, double-float alongside FP16) agree to 1e-8."""
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, 0.5, seed=2)
    b = synth.z2_source(dims, seed=3)
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U))
    xs, st = api.multimass_solve(g, [_cuda(b)], MASSES8, api.params(inner_prec=inner))
    xm = [torch.empty_like(xs[0][0]) for _ in MASSES8]
    stm = api.bicgstab_m_solve(g, _cuda(b), xm, MASSES8, api.params(outer_prec="f64" if inner == "f32" else "df"))
    for i, m in enumerate(MASSES8):
        assert st[0][i]["true_relres"] <= TOL, (m, st[0][i])
        x = xs[0][i].cpu().numpy()
        assert O.true_relres(U, dims, b, x, m) <= SLACK * TOL, m
        assert stm[i]["true_relres"] <= TOL and stm[i]["restarts"] == 0, (m, stm[i])
        assert rel(x, xm[i].cpu().numpy()) < 1e-8, m


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    return json.load(open(path)) if os.path.exists(path) else None


def _golden_errors(gold, xs_of_source, masses, label):
    """Relative l2 error at the stored sites of every recorded solution;
    printed per source and mass."""
    sites = torch.from_numpy(np.array(gold["sites"])).cuda()
    errs = {}
    for k, xs in xs_of_source.items():
        rec = gold["sources"].get(str(k))
        if rec is None:
            continue
        for i, m in enumerate(masses):
            want = np.array(rec["x"][i])[..., 0] + 1j * np.array(rec["x"][i])[..., 1]
            got = xs[i][sites].cpu().numpy().reshape(len(gold["sites"]), 12)
            errs[(k, i)] = rel(got, want)
            print(f"{label} source {k} m0 {m:.4f}: solution error vs oracle at {len(gold['sites'])} sites "
                  f"{errs[(k, i)]:.2e}")
    return errs


@pytest.mark.parametrize("outer", ["f64", "df"])
def test_24c64_twelve_point_sources_batched(api, outer):
    """24^3x64, eps 0.5, 12 spin-colour point sources in one batched FP32-inner
    call, 8 masses: oracle full true residual for two sources at every mass,
    sampled oracle residual for all twelve, every solution against the
    oracle's stored solutions."""
    dims = (24, 24, 24, 64)
    U = synth.gauge_field(dims, 0.5, seed=3)
    bs = [synth.point_source(dims, s, c) for s in range(4) for c in range(3)]
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U))
    xs, st = api.multimass_solve(g, [_cuda(b) for b in bs], MASSES8, api.params(inner_prec="f32", outer_prec=outer))
    chk = SampledResidual(dims, U)
    for r, b in enumerate(bs):
        for i, m in enumerate(MASSES8):
            assert st[r][i]["true_relres"] <= TOL, (r, m, st[r][i])
            est, peak = chk(xs[r][i], b, m)
            assert peak <= SLACK * TOL and est <= 1.5 * TOL, (r, m, est, peak)
    for r in (0, 11):
        for i, m in enumerate(MASSES8):
            assert O.true_relres(U, dims, bs[r], xs[r][i].cpu().numpy(), m) <= SLACK * TOL, (r, m)
    # solution error against the oracle's own multi-mass run (tests/golden,
    # written by make_oracle_multimass.py), every recorded source and mass
    gold = _golden("c3_oracle_multimass.json")
    assert gold is not None and tuple(gold["dims"]) == dims and gold["gauge_seed"] == 3
    assert gold["masses"] == MASSES8 and "0" in gold["sources"]
    errs = _golden_errors(gold, {k: xs[k] for k in range(len(bs))}, MASSES8, f"24^3x64 {outer} outer")
    assert len(errs) >= 8 and max(errs.values()) < 1e-8, max(errs.values())
    # double-float BiCGstab-M on source 0 with a Gaussian shadow residual: every
    # shift converges without the single-mass polish and agrees with the
    # single-mass solutions
    xm = [torch.empty_like(xs[0][0]) for _ in MASSES8]
    rh = _cuda(synth.gaussian_source(dims, seed=103))
    stm = api.bicgstab_m_solve(g, _cuda(bs[0]), xm, MASSES8, api.params(shadow=rh))
    for i, m in enumerate(MASSES8):
        assert stm[i]["true_relres"] <= TOL and stm[i]["restarts"] == 0, (m, stm[i])
        assert rel(xm[i].cpu().numpy(), xs[0][i].cpu().numpy()) < 1e-8, m


@pytest.mark.parametrize("outer", ["f64", "df"])
def test_48c96_fp16_inner_three_sources_sixteen_masses(api, outer):
    """48^3x96 (10.6M sites), eps 0.7, three point sources per call in the
    benchmark's solver configuration (spin-colour 0, 5 and 11; FP16-storage
    inner solves refined in FP32 segments, 4 iterations per captured graph,
    the Lagrange guess through the last 6 masses), 16 log-spaced masses
    0.5 * 0.04^(i/15): every mass at 1e-10, checked by the oracle at sampled
    sites, and the solutions against the oracle's stored ones."""
    dims = (48, 48, 48, 96)
    U = synth.gauge_field(dims, 0.7, seed=5)
    ks = [0, 5, 11]
    bs = [synth.point_source(dims, k // 3, k % 3) for k in ks]
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U), precs=(outer, "f32", "f16"))
    prm = api.params(inner_prec="f16", outer_prec=outer, inner_refine=1, graph_iters=4, guess_max=6)
    xs, st = api.multimass_solve(g, [_cuda(b) for b in bs], MASSES16, prm)
    chk = SampledResidual(dims, U)
    for r, b in enumerate(bs):
        for i, m in enumerate(MASSES16):
            assert st[r][i]["true_relres"] <= TOL, (r, m, st[r][i])
            est, peak = chk(xs[r][i], b, m)
            print(f"48^3x96 {outer} outer source {ks[r]} m0 {m:.4f}: iterations {st[r][i]['iterations']}, "
                  f"GPU true relres {st[r][i]['true_relres']:.2e}, oracle sampled {est:.2e}, peak site {peak:.2e}")
            assert peak <= SLACK * TOL and est <= 1.5 * TOL, (r, m, est, peak)
    gold = _golden("c5_oracle_multimass.json")
    if gold is None:
        pytest.skip("no stored oracle solutions for 48^3x96")
    assert tuple(gold["dims"]) == dims and gold["gauge_seed"] == 5
    errs = _golden_errors(gold, {k: xs[r] for r, k in enumerate(ks)}, MASSES16, f"48^3x96 {outer} outer")
    assert errs and max(errs.values()) < 1e-8, max(errs.values())
