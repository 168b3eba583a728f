"""GPU solver parity: every mass reaches FP64 true relative residual <= 1e-10
and the solution agrees with the FP64 oracle to 1e-8 (relative l2)."""
import numpy as np
import pytest
import torch

from helpers import rel
from oracle import oracle as O
from paper_1103_5103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1103_5103_gb300 import api as A
    return A


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gauge(api, dims, eps, seed, precs=("f64", "f32", "f16", "df")):
    U = synth.gauge_field(dims, eps, seed=seed)
    lat = api.Lattice(dims)
    return U, lat, api.Gauge(lat, _cuda(U), precs=precs)


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
@pytest.mark.parametrize("mode", ["graph", "host"])
@pytest.mark.parametrize("outer", ["df", "f64"])
def test_bicgstab_solve_vs_oracle(api, inner, mode, outer):
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.3, 11)
    b = synth.z2_source(dims, seed=12)
    m0 = 0.1
    x = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    prm = api.params(inner_prec=inner, mode=api.MODE_GRAPH if mode == "graph" else api.MODE_HOST,
                     outer_prec=outer)
    st = api.bicgstab_solve(g, _cuda(b), x, m0, prm)
    assert st["status"] == 0 and st["true_relres"] <= 1e-10, st
    ref, _ = O.eo_solve(U, dims, b, m0, tol=1e-13)
    assert rel(x.cpu().numpy(), ref) < 1e-8
    assert O.true_relres(U, dims, b, x.cpu().numpy(), m0) <= 1.1e-10


@pytest.mark.parametrize("inner", ["f32", "f16"])
@pytest.mark.parametrize("outer", ["df", "f64"])
def test_multimass_c1_config(api, inner, outer):
    """8^4, eps 0.3, point source, masses {0.5, 0.3, 0.2, 0.1}."""
    dims = (8, 8, 8, 8)
    U, lat, g = _gauge(api, dims, 0.3, 1)
    b = synth.point_source(dims)
    masses = [0.5, 0.3, 0.2, 0.1]
    xs, stats = api.multimass_solve(g, [_cuda(b)], masses, api.params(inner_prec=inner, outer_prec=outer))
    ref, _ = O.multimass_solve(U, dims, b, masses, tol=1e-12)
    for i, m in enumerate(masses):
        st = stats[0][i]
        assert st["status"] == 0 and st["true_relres"] <= 1e-10, st
        assert abs(st["mass"] - m) == 0
        assert rel(xs[0][i].cpu().numpy(), ref[i]) < 1e-8


def test_multimass_batched_rhs_and_guesses(api):
    """Several sources in one call, unordered masses, zero vs polynomial guess."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 21)
    bs = [synth.point_source(dims, 0, 0), synth.point_source(dims, 2, 1), synth.z2_source(dims, 22)]
    masses = [0.2, 0.4, 0.05, 0.3]
    for guess in (api.GUESS_ZERO, api.GUESS_POLY):
        xs, stats = api.multimass_solve(g, [_cuda(b) for b in bs], masses, api.params(guess=guess))
        for r, b in enumerate(bs):
            for i, m in enumerate(masses):
                assert stats[r][i]["status"] == 0 and stats[r][i]["true_relres"] <= 1e-10
                ref, _ = O.eo_solve(U, dims, b, m, tol=1e-13)
                assert rel(xs[r][i].cpu().numpy(), ref) < 1e-8


def test_multimass_guess_reduces_iterations(api):
    dims = (8, 8, 8, 8)
    U, lat, g = _gauge(api, dims, 0.3, 31)
    b = _cuda(synth.z2_source(dims, 32))
    masses = [0.40, 0.35, 0.30, 0.25, 0.20]
    _, s0 = api.multimass_solve(g, [b], masses, api.params(guess=api.GUESS_ZERO, inner_prec="f64"))
    _, s1 = api.multimass_solve(g, [b], masses, api.params(guess=api.GUESS_POLY, inner_prec="f64"))
    it0 = sum(s["iterations"] for s in s0[0])
    it1 = sum(s["iterations"] for s in s1[0])
    assert it1 < it0, (it0, it1)


@pytest.mark.parametrize("outer", ["f64", "df"])
def test_bicgstab_m_vs_oracle(api, outer):
    """BiCGstab-M with FP64 or double-float vectors and hops against the
    oracle's FP64 recursion."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 41, precs=(outer,))
    b = synth.z2_source(dims, 42)
    masses = [0.4, 0.25, 0.1, 0.05]
    xs = [torch.empty((lat.volume, 4, 3), dtype=torch.complex128, device="cuda") for _ in masses]
    stats = api.bicgstab_m_solve(g, _cuda(b), xs, masses, api.params(outer_prec=outer))
    ref, _ = O.bicgstab_m(U, dims, b, masses, tol=1e-12)
    for i, m in enumerate(masses):
        assert stats[i]["true_relres"] <= 1e-10, stats[i]
        assert stats[i]["restarts"] == 0, stats[i]   # no single-mass polish was needed
        assert rel(xs[i].cpu().numpy(), ref[i]) < 1e-8
    # the unshifted (lightest) mass needs the most iterations; heavier ones freeze earlier
    its = [stats[i]["iterations"] for i in range(len(masses))]
    assert its[3] == max(its) and its[0] <= its[3]
    # the library iterates the unshifted system to tol/2 (iterated/true residual
    # gap); the oracle's recursion run to the same target needs the same count
    _, ost = O.bicgstab_m(U, dims, b, masses, tol=0.5e-10)
    assert abs(its[3] - ost["iterations"][3]) <= 1, (its, ost["iterations"])


def test_solver_rejects_bad_arguments(api):
    dims = (4, 4, 4, 4)
    U, lat, g = _gauge(api, dims, 0.3, 1, precs=("f64", "f32", "df"))
    b = _cuda(synth.point_source(dims))
    with pytest.raises(api.WilsonError):
        api.multimass_solve(g, [b], [0.1, 0.1], api.params())           # duplicate masses
    with pytest.raises(api.WilsonError):
        api.multimass_solve(g, [b], [0.1], api.params(inner_prec="f16"))  # no FP16 links
    with pytest.raises(api.WilsonError):
        api.multimass_solve(g, [b], [-4.5], api.params())                 # 2 m0 + 8 <= 0
    with pytest.raises(api.WilsonError):
        api.multimass_solve(g, [b], [0.1], api.params(inner_prec="df"))   # DF is an outer precision only


def test_noconv_status_keeps_last_iterate(api):
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.3, 51)
    b = _cuda(synth.z2_source(dims, 52))
    x = torch.zeros_like(b)
    st = api.bicgstab_solve(g, b, x, 0.05, api.params(max_iter=3, inner_prec="f64", graph_iters=1), check=False)
    assert st["call_status"] == api.WL_ERR_NOCONV
    assert 0 < st["true_relres"] < 1.0


@pytest.mark.parametrize("mode", ["graph", "host"])
def test_profiling_counts_hop_launches(api, mode):
    """Live hop timing: events around the first hop of each iteration, in
    captured graphs too; no error leaks into later calls."""
    dims = (8, 8, 8, 8)
    U, lat, g = _gauge(api, dims, 0.3, 61, precs=("f64", "f32", "df"))
    b = _cuda(synth.z2_source(dims, 62))
    api.profile_enable(g, True)
    n0 = api.launch_count()
    prm = api.params(mode=api.MODE_GRAPH if mode == "graph" else api.MODE_HOST)
    xs, stats = api.multimass_solve(g, [b, b], [0.3, 0.1], prm)
    both = api.profile_read(g)
    prof, outer = both["f32"], both["outer"]
    api.profile_enable(g, False)
    iters = stats[0][0]["iterations"] + stats[0][1]["iterations"]
    assert 0 < prof["launches"] <= iters
    assert prof["launches"] >= iters // 2
    assert 0 < prof["ms"] / prof["launches"] < 10.0
    assert prof["site_rhs"] == 2 * prof["sites"] == 2 * prof["launches"] * lat.volume // 2
    # the outer residual hop: one timed launch per hop-based check, covering
    # the rhs still iterating (at least one check per mass, each with one or
    # both rhs)
    restarts = sum(st["restarts"] for st in stats[0])
    assert 2 <= outer["launches"] and restarts <= outer["launches"] <= restarts + 2
    assert outer["sites"] == outer["launches"] * lat.volume // 2
    assert outer["sites"] <= outer["site_rhs"] <= 2 * outer["sites"]
    assert 0 < outer["ms"] / outer["launches"] < 10.0
    assert api.launch_count() - n0 >= 7 * prof["launches"]
    # a following solve is unaffected
    _, st2 = api.multimass_solve(g, [b], [0.2], api.params())
    assert st2[0][0]["status"] == 0


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_persistent_mode_vs_oracle(api, inner):
    """WL_MODE_PERSISTENT: one cooperative kernel per inner solve, same answers."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.3, 11)
    b = synth.z2_source(dims, seed=12)
    x = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
    st = api.bicgstab_solve(g, _cuda(b), x, 0.1, api.params(inner_prec=inner, mode=api.MODE_PERSISTENT))
    assert st["status"] == 0 and st["true_relres"] <= 1e-10, st
    ref, _ = O.eo_solve(U, dims, b, 0.1, tol=1e-13)
    assert rel(x.cpu().numpy(), ref) < 1e-8


def test_persistent_multimass_batched(api):
    dims = (8, 8, 8, 8)
    U, lat, g = _gauge(api, dims, 0.3, 1)
    bs = [synth.point_source(dims, s, c) for s in range(2) for c in range(2)]
    masses = [0.5, 0.3, 0.2, 0.1]
    xs, stats = api.multimass_solve(g, [_cuda(b) for b in bs], masses, api.params(mode=api.MODE_PERSISTENT))
    xg, _ = api.multimass_solve(g, [_cuda(b) for b in bs], masses, api.params(mode=api.MODE_GRAPH))
    for r in range(len(bs)):
        for i in range(len(masses)):
            assert stats[r][i]["status"] == 0 and stats[r][i]["true_relres"] <= 1e-10
            assert rel(xs[r][i].cpu().numpy(), xg[r][i].cpu().numpy()) < 1e-8


def test_persistent_barrier_wait_is_bounded(api):
    """A withheld barrier arrival ends the persistent kernel with WL_ERR_TIMEOUT
    after the wait limit; the context stays usable for the next solve."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.3, 5)
    assert api.persistent_selftest(g, "f32", inject_missing_arrival=False, wait_limit_s=0.5) == api.WL_OK
    assert api.persistent_selftest(g, "f32", inject_missing_arrival=True, wait_limit_s=0.05) == api.WL_ERR_TIMEOUT
    b = _cuda(synth.z2_source(dims, 6))
    x = torch.zeros_like(b)
    st = api.bicgstab_solve(g, b, x, 0.2, api.params(mode=api.MODE_PERSISTENT))
    assert st["status"] == 0 and st["true_relres"] <= 1e-10


def test_f16_inner_with_source_entries_below_float_range(api):
    """A source with entries in the FP32 denormal range (as a point-source
    residual far from the source on a large lattice) must not break the
    FP16-storage inner solve."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.3, seed=1)
    b = synth.point_source(dims) + 1e-40 * synth.gaussian_source(dims, seed=12)
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U))
    x = torch.zeros_like(_cuda(b))
    st = api.bicgstab_solve(g, _cuda(b), x, 0.1, api.params(inner_prec="f16"))
    assert st["status"] == api.WL_OK and st["true_relres"] <= 1e-10, st
    assert O.true_relres(U, dims, b, x.cpu().numpy(), 0.1) <= 1.02e-10


@pytest.mark.parametrize("outer", ["f64", "df"])
def test_bicgstab_m_point_source_with_gaussian_shadow(api, outer):
    """Point source, shadow residual = Gaussian noise (passed to both sides):
    the shifted solutions match the oracle's, with the same iteration count,
    and no mass needs the single-mass polish."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 43, precs=(outer,))
    b = synth.point_source(dims, 1, 2)
    rh = synth.gaussian_source(dims, seed=44)
    masses = [0.4, 0.2, 0.05]
    xs = [torch.empty((lat.volume, 4, 3), dtype=torch.complex128, device="cuda") for _ in masses]
    stats = api.bicgstab_m_solve(g, _cuda(b), xs, masses, api.params(shadow=_cuda(rh), outer_prec=outer))
    ref, ost = O.bicgstab_m(U, dims, b, masses, tol=0.5e-10, rhat=rh)
    assert ost["status"] == O.OK
    for i, m in enumerate(masses):
        assert stats[i]["true_relres"] <= 1e-10 and stats[i]["restarts"] == 0, stats[i]
        assert rel(xs[i].cpu().numpy(), ref[i]) < 1e-8
    assert abs(stats[2]["iterations"] - ost["iterations"][2]) <= 1, (stats, ost)


def test_bicgstab_m_point_source_without_shadow_reports_breakdown(api):
    """rhat = b for a point source: <rhat, r_1> = 0, the shifted recurrences
    stop with WL_ERR_BREAKDOWN (as the oracle's do), every mass is then
    polished by single-mass FP64 BiCGstab, and the polish is visible in
    stats.restarts."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 43, precs=("f64",))
    b = synth.point_source(dims)
    masses = [0.4, 0.1]
    _, ost = O.bicgstab_m(U, dims, b, masses, tol=1e-10)
    assert ost["status"] == O.BREAKDOWN
    xs = [torch.empty((lat.volume, 4, 3), dtype=torch.complex128, device="cuda") for _ in masses]
    with pytest.raises(api.WilsonError) as e:
        api.bicgstab_m_solve(g, _cuda(b), xs, masses, api.params(outer_prec="f64"))
    assert e.value.status == api.WL_ERR_BREAKDOWN
    stats = api.bicgstab_m_solve(g, _cuda(b), xs, masses, api.params(outer_prec="f64"), check=False)
    for i, m in enumerate(masses):
        assert stats[i]["restarts"] > 0 and stats[i]["true_relres"] <= 1e-10, stats[i]
        assert O.true_relres(U, dims, b, xs[i].cpu().numpy(), m) <= 1.02e-10


def test_bicgstab_m_needs_links_of_its_precision(api):
    """FP64 BiCGstab-M (the default outer_prec) on a handle with
    double-float links only, and an inner precision as outer_prec, are
    argument errors."""
    dims = (4, 4, 4, 4)
    U, lat, g = _gauge(api, dims, 0.3, 1, precs=("df",))
    b = _cuda(synth.z2_source(dims, 2))
    xs = [torch.empty_like(b) for _ in range(2)]
    for prm in (api.params(), api.params(outer_prec="f32")):
        with pytest.raises(api.WilsonError) as e:
            api.bicgstab_m_solve(g, b, xs, [0.3, 0.1], prm)
        assert e.value.status == api.WL_ERR_ARG


@pytest.mark.parametrize("guess,guess_max", [("poly", 0), ("poly", 2), ("ssm", 0), ("ssm", 2)])
def test_multimass_guess_iterations_match_oracle(api, guess, guess_max):
    """FP64 inner and outer: with the same initial guess (Lagrange or
    solution-space minimisation, from all or the last two solutions) the
    library and the oracle need the same iterations per mass, and reach the
    same solutions.  A wrong guess coefficient would show here."""
    dims = (8, 8, 8, 8)
    U, lat, g = _gauge(api, dims, 0.3, 31)
    b = synth.z2_source(dims, 33)
    masses = [0.40, 0.35, 0.30, 0.25, 0.20]
    code = {"poly": api.GUESS_POLY, "ssm": api.GUESS_SSM}[guess]
    xs, st = api.multimass_solve(g, [_cuda(b)], masses,
                                 api.params(guess=code, guess_max=guess_max, inner_prec="f64", outer_prec="f64"))
    ref, ost = O.multimass_solve(U, dims, b, masses, tol=1e-10, guess=guess, guess_max=guess_max)
    for i, m in enumerate(masses):
        assert st[0][i]["true_relres"] <= 1e-10, st[0][i]
        assert rel(xs[0][i].cpu().numpy(), ref[i]) < 1e-8
        assert abs(st[0][i]["iterations"] - ost[i]["iterations"]) <= 2, (m, st[0][i], ost[i])


def test_multimass_ssm_batched_fp32_inner(api):
    """SSM guess with several sources (complex coefficients per source) and
    the FP32 inner solve: every mass converges, fewer iterations than the
    zero guess."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 21)
    bs = [synth.point_source(dims, 0, 0), synth.z2_source(dims, 22), synth.gaussian_source(dims, 23)]
    masses = [0.2, 0.4, 0.05, 0.3, 0.1]
    its = {}
    for guess in (api.GUESS_ZERO, api.GUESS_SSM):
        xs, stats = api.multimass_solve(g, [_cuda(b) for b in bs], masses, api.params(guess=guess))
        its[guess] = sum(stats[r][i]["iterations"] for r in range(3) for i in range(len(masses)))
        for r, b in enumerate(bs):
            for i, m in enumerate(masses):
                assert stats[r][i]["status"] == 0 and stats[r][i]["true_relres"] <= 1e-10
                ref, _ = O.eo_solve(U, dims, b, m, tol=1e-13)
                assert rel(xs[r][i].cpu().numpy(), ref) < 1e-8
    assert its[api.GUESS_SSM] < its[api.GUESS_ZERO], its


def test_critical_mass_estimate(api):
    """m_c from the rightmost eigenvalue of the library's FP64 hop: the free
    field's closed form cos(pi/T) - 1, and a random field's dense spectrum."""
    pytest.importorskip("scipy")
    from paper_1103_5103_gb300.mass_sets import critical_mass
    dims = (4, 4, 4, 8)
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(synth.unit_gauge_field(dims)), precs=("f64",))
    mc, ok, _ = critical_mass(g, tol=1e-12)
    assert ok and abs(mc - (np.cos(np.pi / 8) - 1)) < 1e-8
    U = synth.gauge_field(dims, 0.5, seed=5)
    g = api.Gauge(lat, _cuda(U), precs=("f64",))
    dense = np.linalg.eigvals(O.dense_operator(O.OP_HOP, U, dims))
    mc, ok, _ = critical_mass(g, tol=1e-12)
    assert ok and abs(mc - (dense.real.max() / 2 - 4)) < 1e-8


@pytest.mark.parametrize("inner", ["f32", "f16"])
@pytest.mark.parametrize("mode", ["graph", "host"])
def test_reliable_updates_vs_oracle(api, inner, mode):
    """Reliable updates instead of restarted defect correction: the inner
    BiCGstab keeps its shadow residual and direction across the FP64-class
    residual replacements, and still reaches the oracle's solution."""
    dims = (8, 8, 8, 8)
    U, lat, g = _gauge(api, dims, 0.3, 11)
    b = synth.z2_source(dims, seed=12)
    for m0 in (0.3, 0.05):
        x = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
        prm = api.params(inner_prec=inner, reliable=1,
                         mode=api.MODE_GRAPH if mode == "graph" else api.MODE_HOST)
        st = api.bicgstab_solve(g, _cuda(b), x, m0, prm)
        assert st["status"] == 0 and st["true_relres"] <= 1e-10, st
        ref, _ = O.eo_solve(U, dims, b, m0, tol=1e-13)
        assert rel(x.cpu().numpy(), ref) < 1e-8
        assert O.true_relres(U, dims, b, x.cpu().numpy(), m0) <= 1.1e-10


def test_reliable_updates_multimass_batched(api):
    """Several sources and masses with the FP16 inner solve and reliable
    updates: every solution converges to the oracle's."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 21)
    bs = [synth.point_source(dims, 0, 0), synth.z2_source(dims, 22), synth.gaussian_source(dims, 23)]
    masses = [0.2, 0.4, 0.05]
    xs, stats = api.multimass_solve(g, [_cuda(b) for b in bs], masses, api.params(inner_prec="f16", reliable=1))
    for r, b in enumerate(bs):
        for i, m in enumerate(masses):
            assert stats[r][i]["status"] == 0 and stats[r][i]["true_relres"] <= 1e-10, stats[r][i]
            ref, _ = O.eo_solve(U, dims, b, m, tol=1e-13)
            assert rel(xs[r][i].cpu().numpy(), ref) < 1e-8


def test_pinned_host_sources_and_solutions(api):
    """Canonical sources and solutions in page-locked host memory: the layout
    kernels read and write them directly, with results identical to the
    device-memory call."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 21)
    bs = [synth.point_source(dims, 1, 1), synth.z2_source(dims, 24)]
    masses = [0.3, 0.1]
    xd, sd = api.multimass_solve(g, [_cuda(b) for b in bs], masses)
    bh = [torch.from_numpy(b).pin_memory() for b in bs]
    xh = [[torch.empty_like(b).pin_memory() for _ in masses] for b in bh]
    _, sh = api.multimass_solve(g, bh, masses, xs=xh)
    torch.cuda.synchronize()
    for r in range(len(bs)):
        for i in range(len(masses)):
            assert torch.equal(xh[r][i], xd[r][i].cpu()), (r, i)
            assert sh[r][i]["iterations"] == sd[r][i]["iterations"]
    out = torch.empty_like(bh[0]).pin_memory()
    api.wilson_dslash(g, bh[1], out, 0.12, "f64", api.OP_M)
    torch.cuda.synchronize()
    assert rel(out.numpy(), O.apply(O.OP_MK, U, dims, bs[1], 0.12)) < 1e-12
    with pytest.raises(ValueError):
        api.multimass_solve(g, [torch.from_numpy(bs[0])], masses)   # pageable host memory is refused


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
@pytest.mark.parametrize("mode", ["graph", "host"])
def test_cg_normal_equations_inner_solver(api, inner, mode):
    """CG on the normal equations M^dag M e = M^dag r as the inner solver of
    the defect correction (the dagger hops are gamma5-conjugated): the same
    solution as the oracle's BiCGstab solve."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.3, 11)
    b = synth.z2_source(dims, seed=12)
    for m0 in (0.3, 0.05):
        x = torch.zeros((lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
        prm = api.params(inner_prec=inner, inner_solver=api.SOLVER_CG,
                         mode=api.MODE_GRAPH if mode == "graph" else api.MODE_HOST)
        st = api.bicgstab_solve(g, _cuda(b), x, m0, prm)
        assert st["status"] == 0 and st["true_relres"] <= 1e-10, st
        ref, _ = O.eo_solve(U, dims, b, m0, tol=1e-13)
        assert rel(x.cpu().numpy(), ref) < 1e-8


def test_cg_multimass_batched_and_rejected_combinations(api):
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 21)
    bs = [synth.point_source(dims, 0, 0), synth.z2_source(dims, 22)]
    masses = [0.2, 0.4, 0.05]
    xs, stats = api.multimass_solve(g, [_cuda(b) for b in bs], masses, api.params(inner_solver=api.SOLVER_CG))
    for r, b in enumerate(bs):
        for i, m in enumerate(masses):
            assert stats[r][i]["status"] == 0 and stats[r][i]["true_relres"] <= 1e-10, stats[r][i]
            ref, _ = O.eo_solve(U, dims, b, m, tol=1e-13)
            assert rel(xs[r][i].cpu().numpy(), ref) < 1e-8
    for bad in (dict(reliable=1), dict(mode=api.MODE_PERSISTENT)):
        with pytest.raises(api.WilsonError) as e:
            api.multimass_solve(g, [_cuda(bs[0])], masses, api.params(inner_solver=api.SOLVER_CG, **bad))
        assert e.value.status == api.WL_ERR_ARG


def test_multimass_mass_count_edges(api):
    """One mass (no guess to build), the maximum of sixteen (a Lagrange guess
    through fifteen solutions, 31 inputs to one combination), and seventeen,
    which is refused."""
    dims = (4, 4, 2, 4)
    U, lat, g = _gauge(api, dims, 0.4, 61)
    b = synth.gaussian_source(dims, seed=62)
    xs, st = api.multimass_solve(g, [_cuda(b)], [0.25])
    assert st[0][0]["true_relres"] <= 1e-10
    assert rel(xs[0][0].cpu().numpy(), O.eo_solve(U, dims, b, 0.25, tol=1e-13)[0]) < 1e-8
    masses = [0.5 * 0.04 ** (i / 15.0) for i in range(16)]
    for guess in (api.GUESS_POLY, api.GUESS_SSM):
        xs, st = api.multimass_solve(g, [_cuda(b)], masses, api.params(guess=guess))
        for i, m in enumerate(masses):
            assert st[0][i]["true_relres"] <= 1e-10, (m, st[0][i])
        for i in (0, 7, 15):
            assert rel(xs[0][i].cpu().numpy(), O.eo_solve(U, dims, b, masses[i], tol=1e-13)[0]) < 1e-8
    with pytest.raises(api.WilsonError) as e:
        api.multimass_solve(g, [_cuda(b)], masses + [0.9])
    assert e.value.status == api.WL_ERR_ARG


def test_gauge_create_rejects_links_off_su3(api):
    """The 12-real formats rebuild the third row of a link from the first
    two, so links off SU(3) are refused: a link scaled by 1.001 (not
    unitary), a U(3) link (det = e^{0.3 i}) and a NaN entry each give
    WL_ERR_ARG; a perturbation at 1e-9 (rounding of stored links) is
    accepted."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, seed=5)
    lat = api.Lattice(dims)
    bad = []
    for k in range(3):
        B = U.copy()
        if k == 0:
            B[1, 17] *= 1.001
        elif k == 1:
            B[2, 40] *= np.exp(0.1j)
        else:
            B[3, 9, 1, 2] = complex(float("nan"), 0.0)
        bad.append(B)
    for B in bad:
        with pytest.raises(api.WilsonError) as e:
            api.Gauge(lat, _cuda(B), precs=("f32",))
        assert e.value.status == api.WL_ERR_ARG
    ok = U + 1e-9 * synth.gauge_field(dims, 0.5, seed=6)
    g = api.Gauge(lat, _cuda(ok), precs=("f32",))
    g.close()


def test_nan_source_breaks_down_alone(api):
    """A source with a NaN entry, batched with a good one: its masses report
    WL_ERR_BREAKDOWN (non-finite residual) while the good source converges
    to 1e-10 at every mass, the same as solved alone."""
    dims = (4, 4, 4, 8)
    U, lat, g = _gauge(api, dims, 0.5, 7, precs=("f64", "f32", "df"))
    good = synth.z2_source(dims, 8)
    nan = synth.z2_source(dims, 9)
    nan[5, 2, 1] = complex(float("nan"), 1.0)
    masses = [0.4, 0.2, 0.1]
    xs, st = api.multimass_solve(g, [_cuda(good), _cuda(nan)], masses, api.params(), check=False)
    for i, m in enumerate(masses):
        assert st[1][i]["status"] == api.WL_ERR_BREAKDOWN, st[1][i]
        assert st[0][i]["status"] == api.WL_OK and st[0][i]["true_relres"] <= 1e-10, st[0][i]
        assert O.true_relres(U, dims, good, xs[0][i].cpu().numpy(), m) <= 1.02e-10
    with pytest.raises(api.WilsonError) as e:
        api.multimass_solve(g, [_cuda(nan)], masses, api.params())
    assert e.value.status == api.WL_ERR_BREAKDOWN


@pytest.mark.parametrize("outer", ["f64", "df"])
def test_full_residual_from_last_check_equals_recomputed(api, outer):
    """The reported full-lattice residual takes its even half from the last
    outer check, b_prec - M_prec x_e (Section 6.2.3: equal to b_e - x_e +
    kappa D_eo x_o up to the rounding of the rebuilt x_o).  Recomputing it
    with the extra hop D_eo x_o (verify_full = 1) gives the same figure to
    well under a percent, the same solutions, and both agree with the
    oracle's full-lattice residual of the returned x."""
    dims = (8, 8, 8, 16)
    U, lat, g = _gauge(api, dims, 0.5, 71, precs=("f64", "f32", "f16", "df"))
    bs = [synth.point_source(dims, 1, 1), synth.z2_source(dims, 72)]
    masses = [0.4, 0.2, 0.1]
    res = {}
    for vf in (0, 1):
        xs, st = api.multimass_solve(g, [_cuda(b) for b in bs], masses,
                                     api.params(inner_prec="f16", outer_prec=outer, verify_full=vf))
        res[vf] = (xs, st)
    # double-float residuals carry about 48-bit rounding: a few 1e-15 of
    # ||b||, a few 1e-4 of a 1e-11 residual
    slack = {"f64": 1e-3, "df": 2e-2}[outer]
    for r, b in enumerate(bs):
        for i, m in enumerate(masses):
            a, c = res[0][1][r][i]["true_relres"], res[1][1][r][i]["true_relres"]
            assert 0 < a <= 1e-10 and 0 < c <= 1e-10, (r, m, a, c)
            assert abs(a - c) <= slack * c, (r, m, a, c)
            x0, x1 = res[0][0][r][i].cpu().numpy(), res[1][0][r][i].cpu().numpy()
            assert rel(x1, x0) < 1e-14
            o = O.true_relres(U, dims, b, x0, m)
            assert abs(o - a) <= slack * o, (r, m, o, a)


def test_grid_stride_outer_hops_and_concurrent_handles(api):
    """FP64 residual hops as a grid-stride kernel (outer_blocks_per_sm 1, 2)
    give the solutions of the full-grid launch; and two batches solved at the
    same time on two handles and two streams, from two host threads, give
    the solutions of the same batches solved one after the other."""
    import threading
    dims = (8, 8, 8, 16)
    U, lat, _ = _gauge(api, dims, 0.5, 81, precs=("f64", "f16"))
    bs = [_cuda(synth.point_source(dims, s, 1)) for s in range(4)]
    masses = [0.4, 0.2, 0.1]
    gs = [api.Gauge(lat, _cuda(U), precs=("f64", "f16")) for _ in range(2)]
    ref = []
    for k in range(2):
        ref.append(api.multimass_solve(gs[0], bs[2 * k:2 * k + 2], masses, api.params(inner_prec="f16"))[0])
    for ob in (1, 2):
        xs, st = api.multimass_solve(gs[0], bs[0:2], masses, api.params(inner_prec="f16", outer_blocks_per_sm=ob))
        for r in range(2):
            for i in range(len(masses)):
                assert st[r][i]["true_relres"] <= 1e-10
                assert rel(xs[r][i].cpu().numpy(), ref[0][r][i].cpu().numpy()) < 1e-14, (ob, r, i)
    streams = [torch.cuda.Stream() for _ in range(2)]
    out = [None, None]

    def work(k):
        out[k] = api.multimass_solve(gs[k], bs[2 * k:2 * k + 2], masses,
                                     api.params(inner_prec="f16", outer_blocks_per_sm=1), stream=streams[k])
    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    for k in range(2):
        xs, st = out[k]
        for r in range(2):
            for i, m in enumerate(masses):
                assert st[r][i]["status"] == api.WL_OK and st[r][i]["true_relres"] <= 1e-10
                assert rel(xs[r][i].cpu().numpy(), ref[k][r][i].cpu().numpy()) < 1e-14, (k, r, i)
                assert O.true_relres(U, dims, bs[2 * k + r].cpu().numpy(), xs[r][i].cpu().numpy(), m) <= 1.02e-10


def test_fp32_refined_fp16_inner_solve(api):
    """FP16 inner solves run as FP16 segments with the inner residual
    recomputed in FP32 between them (inner_refine): every mass still reaches
    the 1e-10 true residual and the oracle's solution, with no more outer
    (FP64) checks than one FP16 solve per outer step takes; without FP32
    links on the handle the option is refused."""
    dims = (8, 8, 8, 16)
    U, lat, g = _gauge(api, dims, 0.5, 91, precs=("f64", "f32", "f16"))
    bs = [synth.point_source(dims, 0, 2), synth.z2_source(dims, 92)]
    masses = [0.4, 0.2, 0.1, 0.05]
    res = {}
    for rf in (0, 1):
        res[rf] = api.multimass_solve(g, [_cuda(b) for b in bs], masses,
                                      api.params(inner_prec="f16", inner_refine=rf))
    refs = [O.multimass_solve(U, dims, b, masses, tol=1e-12)[0] for b in bs]
    for r, b in enumerate(bs):
        for i, m in enumerate(masses):
            st0, st1 = res[0][1][r][i], res[1][1][r][i]
            assert st1["status"] == api.WL_OK and st1["true_relres"] <= 1e-10, st1
            assert st1["restarts"] <= st0["restarts"], (r, m, st0, st1)
            x = res[1][0][r][i].cpu().numpy()
            assert rel(x, refs[r][i]) < 1e-8, (r, m)
            assert O.true_relres(U, dims, b, x, m) <= 1.02e-10
    g16 = api.Gauge(lat, _cuda(U), precs=("f64", "f16"))
    with pytest.raises(api.WilsonError) as e:
        api.multimass_solve(g16, [_cuda(bs[0])], masses, api.params(inner_prec="f16", inner_refine=1))
    assert e.value.status == api.WL_ERR_ARG
