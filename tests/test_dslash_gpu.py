"""GPU parity of the hop / M / M_prec kernels against the FP64 oracle, through
the C ABI (wilson_dslash, wilson_dslash_dag, wilson_hop, spinor import/export).
Tolerances (relative l2): FP64 1e-12, FP32 1e-6, FP16 storage 5e-3."""
import numpy as np
import pytest
import torch

from helpers import TOL, rel
from oracle import oracle as O
from paper_1103_5103_gb300 import synth

pytestmark = pytest.mark.gpu

LATTICES = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 4, 4, 8), (6, 4, 4, 8), (8, 8, 8, 8), (4, 6, 2, 10)]


@pytest.fixture(scope="module")
def api():
    from paper_1103_5103_gb300 import api as A
    return A


def _field(dims, kind, seed=1):
    return synth.unit_gauge_field(dims) if kind == "free" else synth.gauge_field(dims, 0.5, seed=seed)


def _setup(api, dims, kind, antiperiodic=True, precs=("f64", "f32", "f16", "df")):
    U = _field(dims, kind)
    lat = api.Lattice(dims, antiperiodic)
    g = api.Gauge(lat, torch.from_numpy(U).cuda(), precs=precs)
    return U, lat, g


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("kind", ["free", "random"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df"])
def test_dslash_ops_vs_oracle(api, dims, kind, prec):
    U, lat, g = _setup(api, dims, kind)
    psi = synth.gaussian_source(dims, seed=5)
    kappa = 0.123
    dpsi = _cuda(psi)
    out = torch.empty_like(dpsi)
    for op, okind, par in [(api.OP_HOP, O.OP_HOP, 0.0), (api.OP_M, O.OP_MK, kappa), (api.OP_MPREC, O.OP_MPREC, kappa)]:
        for dag in (False, True):
            want = O.apply(okind, U, dims, psi, par, dagger=dag)
            if op == api.OP_MPREC:
                src = psi.copy()
                src[O.parity_mask(dims)] = 0
                want = O.apply(okind, U, dims, src, par, dagger=dag)
            f = api.wilson_dslash_dag if dag else api.wilson_dslash
            f(g, dpsi, out, kappa, prec, op)
            torch.cuda.synchronize()
            err = rel(out.cpu().numpy(), want)
            assert err < TOL[prec], (op, dag, err)


@pytest.mark.parametrize("antiperiodic", [True, False])
def test_boundary_conditions(api, antiperiodic):
    dims = (4, 4, 4, 6)
    U, lat, g = _setup(api, dims, "random", antiperiodic)
    psi = synth.z2_source(dims, seed=3)
    out = torch.empty((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    api.wilson_dslash(g, _cuda(psi), out, 0.11, "f64", api.OP_M)
    want = O.apply(O.OP_MK, U, dims, psi, 0.11, antiperiodic=antiperiodic)
    assert rel(out.cpu().numpy(), want) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df"])
def test_internal_layout_roundtrip(api, prec):
    dims = (6, 4, 4, 8)
    lat = api.Lattice(dims)
    psi = synth.gaussian_source(dims, seed=7)
    d = _cuda(psi)
    back = torch.zeros_like(d)
    for par in (0, 1):
        buf = lat.new_internal(prec)
        lat.spinor_import(d, buf, prec, par)
        lat.spinor_export(buf, back, prec, par)
    torch.cuda.synchronize()
    err = rel(back.cpu().numpy(), psi)
    if prec == "f64":
        assert err == 0.0
    else:
        assert err < {"df": 1e-14, "f32": 1e-7, "f16": 1e-3}[prec], err


def test_double_float_and_fp32_export_is_exact(api):
    """Import splits a double into hi = fl32(d), lo = fl32(d - hi) and
    renormalises; export returns hi + lo in FP64, which is exact.  The round
    trip equals the same float arithmetic done in numpy, bit for bit, for
    normal, zero, negative-zero, subnormal-float and extreme values."""
    dims = (2, 2, 2, 2)
    lat = api.Lattice(dims)
    V = lat.volume
    rng = np.random.default_rng(3)
    special = np.array([0.0, -0.0, 1.0, -2.5, 1.0 / 3.0, 1e-40, -3e-42, 1e-38, 3.0e38, -1.17549435e-38,
                        np.pi * 1e20, np.e * 1e-20])
    vals = np.concatenate([special, rng.standard_normal(12 * V * 2 - len(special)) * 10.0 ** rng.integers(-30, 30, 12 * V * 2 - len(special))])
    psi = (vals[0::2] + 1j * vals[1::2]).reshape(V, 4, 3)
    d = _cuda(psi)
    for prec in ("df", "f32"):
        back = torch.zeros_like(d)
        for par in (0, 1):
            buf = lat.new_internal(prec)
            lat.spinor_import(d, buf, prec, par)
            lat.spinor_export(buf, back, prec, par)
        got = back.cpu().numpy().view(np.float64).reshape(-1)
        x = psi.view(np.float64).reshape(-1)
        hi = x.astype(np.float32)
        if prec == "df":
            lo = (x - hi.astype(np.float64)).astype(np.float32)
            s = (hi + lo).astype(np.float32)
            lo = (lo - (s - hi)).astype(np.float32)
            want = s.astype(np.float64) + lo.astype(np.float64)
        else:
            want = hi.astype(np.float64)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), prec


def test_f16_sites_below_float_range_store_as_zero(api):
    """FP16 storage scales each site by its largest entry.  Sites whose
    entries are all below the smallest normal float (here 1e-40, an FP32
    denormal) are stored as zero, not as NaN; sites at 1e-30 and at 1 keep
    FP16 accuracy relative to themselves; the operator stays finite."""
    dims = (6, 4, 4, 8)
    U, lat, g = _setup(api, dims, "random")
    psi = synth.gaussian_source(dims, seed=7)
    n = np.arange(lat.volume)
    scale = np.where(n % 3 == 0, 1e-40, np.where(n % 3 == 1, 1e-30, 1.0))
    psi = psi * scale[:, None, None]
    d = _cuda(psi)
    back = torch.zeros_like(d)
    for par in (0, 1):
        buf = lat.new_internal("f16")
        lat.spinor_import(d, buf, "f16", par)
        lat.spinor_export(buf, back, "f16", par)
    b = back.cpu().numpy()
    assert np.all(np.isfinite(b))
    assert np.all(b[n % 3 == 0] == 0)
    for k in (1, 2):
        s = n % 3 == k
        err = np.linalg.norm((b[s] - psi[s]).reshape(s.sum(), -1), axis=1)
        assert np.all(err <= 2e-3 * np.linalg.norm(psi[s].reshape(s.sum(), -1), axis=1))
    out = torch.empty_like(d)
    api.wilson_dslash(g, d, out, 0.12, "f16", api.OP_M)
    o = out.cpu().numpy()
    assert np.all(np.isfinite(o))
    assert rel(o, O.apply(O.OP_MK, U, dims, psi, 0.12)) < TOL["f16"]


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df"])
@pytest.mark.parametrize("parity", [0, 1])
def test_wilson_hop_internal_xpay(api, prec, parity):
    """out_p = x_p + coef * D_{p,1-p} in on internal buffers."""
    dims = (8, 4, 4, 8)
    U, lat, g = _setup(api, dims, "random")
    psi = synth.gaussian_source(dims, seed=8)
    xv = synth.z2_source(dims, seed=9)
    coef = -0.37
    odd = O.parity_mask(dims)
    src = psi.copy()
    src[odd == bool(parity)] = 0                # keep the input parity 1-p only
    want = xv + coef * O.hop(U, dims, src)
    mask_out = odd if parity == 1 else ~odd
    bi, bx, bo = lat.new_internal(prec), lat.new_internal(prec), lat.new_internal(prec)
    lat.spinor_import(_cuda(psi), bi, prec, 1 - parity)
    lat.spinor_import(_cuda(xv), bx, prec, parity)
    api.wilson_hop(g, bi, bo, bx, coef, prec, parity)
    out = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    lat.spinor_export(bo, out, prec, parity)
    torch.cuda.synchronize()
    err = rel(out.cpu().numpy()[mask_out], want[mask_out])
    assert err < TOL[prec], err


def test_dslash_rejects_bad_arguments(api):
    dims = (4, 4, 4, 4)
    U, lat, g = _setup(api, dims, "free", precs=("f32",))
    d = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    o = torch.zeros_like(d)
    with pytest.raises(api.WilsonError) as e:
        api.wilson_dslash(g, d, o, 0.1, "f64", api.OP_M)    # no FP64 links in this handle
    assert e.value.status == api.WL_ERR_ARG
    with pytest.raises(api.WilsonError):
        api.wilson_dslash(g, d, d, 0.1, "f32", api.OP_M)    # aliasing
    with pytest.raises(api.WilsonError):
        api.wilson_dslash(g, d, o, 0.1, "f32", 7)           # bad operator id


def test_large_lattice_sampled_sites(api):
    """16^3 x 32 FP32 M: compare sampled output sites with the oracle
    computed site by site on a local patch."""
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, 0.5, seed=2)
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U), precs=("f32",))
    psi = synth.gaussian_source(dims, seed=4)
    out = torch.empty((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    api.wilson_dslash(g, _cuda(psi), out, 0.124, "f32", api.OP_M)
    full = O.apply(O.OP_MK, U, dims, psi, 0.124)
    o = out.cpu().numpy()
    rng = np.random.default_rng(0)
    sites = rng.integers(0, lat.volume, size=2000)
    err = rel(o[sites], full[sites])
    assert err < 1e-6


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("rhs_block", [1, 2, 4])
@pytest.mark.parametrize("nrhs", [1, 3, 5])
def test_hop_multi_rhs(api, prec, rhs_block, nrhs):
    """wilson_hop_multi: every rhs of a batch (ragged against the rhs block)
    matches the oracle hop of that rhs."""
    dims = (4, 6, 4, 8)
    U, lat, g = _setup(api, dims, "random")
    odd = O.parity_mask(dims)
    stride = (lat.spinor_bytes(prec) + 255) // 256 * 256
    a = torch.empty(stride * nrhs, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    xb = torch.empty_like(a)
    srcs = [synth.gaussian_source(dims, 100 + r) for r in range(nrhs)]
    xvs = [synth.z2_source(dims, 200 + r) for r in range(nrhs)]
    for r in range(nrhs):
        lat.spinor_import(_cuda(srcs[r]), a[r * stride:(r + 1) * stride], prec, 0)
        lat.spinor_import(_cuda(xvs[r]), xb[r * stride:(r + 1) * stride], prec, 1)
    api.hop_batch(g, a, b, nrhs, stride, 0.5, prec, 1, rhs_block, x=xb)
    for r in range(nrhs):
        out = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
        lat.spinor_export(b[r * stride:(r + 1) * stride], out, prec, 1)
        src = srcs[r].copy()
        src[odd] = 0
        want = xvs[r] + 0.5 * O.hop(U, dims, src)
        assert rel(out.cpu().numpy()[odd], want[odd]) < TOL[prec], r


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df"])
@pytest.mark.parametrize("dims", [(8, 4, 4, 8), (6, 4, 2, 10)])
def test_every_hop_variant_and_autotune(api, prec, dims):
    """Every autotuner variant computes the same hop; wl_autotune picks one of
    them.  On 6x4x2x10 (120 sites per parity) the paired-site variants end on
    a half-filled pair tile, and the TMA variants, which need X/2 a multiple
    of 4, refuse the lattice."""
    U, lat, g = _setup(api, dims, "random")
    nrhs = 5
    odd = O.parity_mask(dims)
    stride = (lat.spinor_bytes(prec) + 255) // 256 * 256
    a = torch.empty(stride * nrhs, dtype=torch.uint8, device="cuda")
    srcs = [synth.gaussian_source(dims, 300 + r) for r in range(nrhs)]
    for r in range(nrhs):
        lat.spinor_import(_cuda(srcs[r]), a[r * stride:(r + 1) * stride], prec, 0)
    for v in api.HOP_VARIANTS[prec]:
        b = torch.zeros_like(a)
        if v >= 9000 and (dims[0] // 2) % 4:
            with pytest.raises(api.WilsonError) as e:
                api.hop_batch(g, a, b, nrhs, stride, 1.0, prec, 1, -v)
            assert e.value.status == api.WL_ERR_ARG
            continue
        api.hop_batch(g, a, b, nrhs, stride, 1.0, prec, 1, -v)
        for r in range(nrhs):
            out = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
            lat.spinor_export(b[r * stride:(r + 1) * stride], out, prec, 1)
            src = srcs[r].copy()
            src[odd] = 0
            want = O.hop(U, dims, src)
            assert rel(out.cpu().numpy()[odd], want[odd]) < TOL[prec], (v, r)
    v, us = api.autotune(g, prec, nrhs)
    assert v in api.HOP_VARIANTS[prec] and us > 0
    assert api.autotune(g, prec, nrhs)[0] == v          # cached


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("dims", [(8, 12, 6, 10), (16, 8, 4, 6)])
def test_tma_staged_hop_matches_register_hop(api, prec, dims):
    """The TMA-staged hop (variants 9000 + rhs per tile: links and spinor
    rows copied into shared memory by cp.async.bulk.tensor) gives, element
    for element, the result of the register kernel for several row blocks
    per slice, rhs counts that leave a ragged last group, both output
    parities and the xpay epilogue; against the oracle too; and no bounded
    wait gives up.  Lattices with X/2 not a multiple of 4 are refused."""
    U, lat, g = _setup(api, dims, "random", precs=(prec,))
    odd = O.parity_mask(dims)
    stride = (lat.spinor_bytes(prec) + 255) // 256 * 256
    for nrhs in (1, 3, 7):
        a = torch.empty(stride * nrhs, dtype=torch.uint8, device="cuda")
        xv = torch.empty_like(a)
        srcs = [synth.gaussian_source(dims, 400 + r) for r in range(nrhs)]
        for par in (0, 1):
            for r in range(nrhs):
                lat.spinor_import(_cuda(srcs[r]), a[r * stride:(r + 1) * stride], prec, 1 - par)
                lat.spinor_import(_cuda(srcs[(r + 1) % nrhs]), xv[r * stride:(r + 1) * stride], prec, par)
            mask = odd if par == 1 else ~odd

            def export(buf, r):
                out = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
                lat.spinor_export(buf[r * stride:(r + 1) * stride], out, prec, par)
                return out.cpu().numpy()[mask]
            want = torch.zeros_like(a)
            api.hop_batch(g, a, want, nrhs, stride, 0.25, prec, par, -101, x=xv)
            for v in (9001, 9002, 9004, 9102, 9104):
                got = torch.zeros_like(a)
                api.hop_batch(g, a, got, nrhs, stride, 0.25, prec, par, -v, x=xv)
                for r in range(nrhs):
                    # same arithmetic; the compiler may contract the row-2
                    # rebuild differently, and FP16 storage rounds at 2^-11
                    assert rel(export(got, r), export(want, r)) < {"f32": 1e-6, "f16": 2e-3}[prec], (v, nrhs, par, r)
            for r in range(nrhs):
                src = srcs[r].copy()
                src[mask] = 0   # the input lives on the other parity
                ref = srcs[(r + 1) % nrhs] + 0.25 * O.hop(U, dims, src)
                assert rel(export(want, r), ref[mask]) < TOL[prec], (nrhs, par, r)
    assert api.wait_faults() == 0
    bad = (6, 4, 4, 4)   # X/2 = 3
    _, lat2, g2 = _setup(api, bad, "random", precs=(prec,))
    s2 = (lat2.spinor_bytes(prec) + 255) // 256 * 256
    a2 = torch.zeros(s2, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.WilsonError) as e:
        api.hop_batch(g2, a2, torch.zeros_like(a2), 1, s2, 1.0, prec, 0, -9001)
    assert e.value.status == api.WL_ERR_ARG
