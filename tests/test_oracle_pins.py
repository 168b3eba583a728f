"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a value printed in the paper (Table 1), or a textbook/library
routine (dense LU, least squares, finite differences).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1103_5103_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(12345)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


# ------------------------------------------------------------ gamma / Table 1

def test_gamma_clifford_and_hermitian():
    g = O.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    # chiral: gamma5 = diag(1, 1, -1, -1)
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]), atol=1e-15)


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_projectors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            head, v1, v2 = line.split("|")
            mu, sgn = head.split()
            rows[(int(mu), sgn)] = (np.array([complex(t) for t in v1.split()]),
                                    np.array([complex(t) for t in v2.split()]))
    return rows


def test_table1_projectors_match_gamma():
    """Table 1: v1 v1^dag + v2 v2^dag = 1 - gamma_mu (T^+) and 1 + gamma_mu (T^-)."""
    g = O.gammas()
    rows = _table1()
    assert len(rows) == 8
    for (mu, sgn), (v1d, v2d) in rows.items():
        v1, v2 = v1d.conj(), v2d.conj()
        P = np.outer(v1, v1d) + np.outer(v2, v2d)
        want = np.eye(4) - g[mu - 1] if sgn == "+" else np.eye(4) + g[mu - 1]
        assert np.allclose(P, want, atol=0), (mu, sgn)


# ------------------------------------------------------- free-field pins

def _plane_wave(dims, k, cvec, u):
    """psi_n = exp(i p.n) c u^T with antiperiodic-time momenta; returns (psi, p)."""
    X, Y, Z, T = dims
    p = np.array([2 * np.pi * k[0] / X, 2 * np.pi * k[1] / Y, 2 * np.pi * k[2] / Z,
                  (2 * k[3] + 1) * np.pi / T])
    xs = synth.lex_coords(dims)
    phase = np.exp(1j * xs @ p)
    psi = phase[:, None, None] * np.einsum("s,c->sc", u, cvec)[None]
    return psi, p, phase


def _Dp(p, g):
    """Momentum-space hop: D(p) = sum_mu [2 cos p_mu - 2 i sin p_mu gamma_mu]
    (right-multiplying the spin row vector)."""
    return sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * g[m] for m in range(4))


@pytest.mark.parametrize("dims", [(4, 2, 2, 4), (2, 2, 2, 2), (4, 4, 2, 6)])
def test_free_field_closed_form(dims):
    g = O.gammas()
    U = synth.unit_gauge_field(dims)
    kap = 0.13
    for trial in range(4):
        k = [int(rng.integers(0, d)) for d in dims]
        u = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        psi, p, phase = _plane_wave(dims, k, c, u)
        out = O.apply(O.OP_MK, U, dims, psi, kap)
        row = u @ (np.eye(4) - kap * _Dp(p, g))           # u^T (1 - kappa D(p))
        want = phase[:, None, None] * np.einsum("s,c->sc", row, c)[None]
        assert _rel(out, want) < 1e-14


def test_free_field_eigenvalues():
    """Eigenvalues of M_k on the free field: 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p),
    each with multiplicity 2 (spin) x 3 (colour) per momentum."""
    dims = (2, 2, 2, 4)
    U = synth.unit_gauge_field(dims)
    kap = 0.11
    M = O.dense_operator(O.OP_MK, U, dims, kap)
    key = lambda z: np.sort_complex(np.round(z.real, 9) + 1j * np.round(z.imag, 9))
    ev = key(np.linalg.eigvals(M))
    want = []
    for kx in range(2):
        for ky in range(2):
            for kz in range(2):
                for kt in range(4):
                    p = np.array([np.pi * kx, np.pi * ky, np.pi * kz, (2 * kt + 1) * np.pi / 4])
                    re = 1 - 2 * kap * np.cos(p).sum()
                    im = 2 * kap * np.sqrt((np.sin(p) ** 2).sum())
                    want += [re + 1j * im] * 6 + [re - 1j * im] * 6
    want = key(np.array(want))
    assert np.allclose(ev, want, atol=1e-8)


def test_constant_abelian_field_closed_form():
    """U_mu = diag(e^{i a}, e^{i b}, e^{-i(a+b)}) per direction: colour c feels
    the momentum p + theta_{mu,c}.  Pins U versus U^dagger on the two hops."""
    dims = (4, 2, 4, 4)
    g = O.gammas()
    V = synth.volume(dims)
    th = rng.uniform(-1, 1, size=(4, 2))
    theta = np.concatenate([th, -th.sum(axis=1, keepdims=True)], axis=1)  # (mu, colour)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    for mu in range(4):
        for c in range(3):
            U[mu, :, c, c] = np.exp(1j * theta[mu, c])
    k = [1, 0, 3, 2]
    u = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    cvec = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    psi, p, phase = _plane_wave(dims, k, cvec, u)
    out = O.hop(U, dims, psi)
    want = np.zeros_like(psi)
    for c in range(3):
        row = u @ _Dp(p + theta[:, c], g)
        want[:, :, c] = phase[:, None] * cvec[c] * row[None, :]
    assert _rel(out, want) < 1e-14


def test_site_sampled_operator_free_field():
    """The site-sampled M_k reproduces the free-field closed form at the sites."""
    dims = (4, 4, 2, 6)
    g = O.gammas()
    U = synth.unit_gauge_field(dims)
    u = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    psi, p, phase = _plane_wave(dims, [1, 3, 1, 2], c, u)
    kap = 0.12
    sites = np.array([0, 5, 17, 63, synth.volume(dims) - 1])
    out = O.apply_mk_sites(U, dims, psi, kap, sites)
    row = u @ (np.eye(4) - kap * _Dp(p, g))
    want = phase[sites][:, None, None] * np.einsum("s,c->sc", row, c)[None]
    assert _rel(out, want) < 1e-14


def test_site_sampled_operator_random_field():
    dims = (4, 2, 2, 6)
    U = synth.gauge_field(dims, 0.7, seed=4)
    psi = synth.gaussian_source(dims, seed=5)
    sites = np.arange(0, synth.volume(dims), 7)
    full = O.apply(O.OP_MK, U, dims, psi, 0.11)
    assert _rel(O.apply_mk_sites(U, dims, psi, 0.11, sites), full[sites]) < 1e-15


# --------------------------------------------------------- gauge-field pins

def test_gauge_covariance():
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, seed=7)
    G = synth.random_gauge_transform(dims, seed=8)
    psi = synth.gaussian_source(dims, seed=9)
    V = synth.volume(dims)
    xs = synth.lex_coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        nb = xs.copy()
        nb[:, mu] = (nb[:, mu] + 1) % dims[mu]
        m = nb[:, 0] + dims[0] * (nb[:, 1] + dims[1] * (nb[:, 2] + dims[2] * nb[:, 3]))
        Ug[mu] = G @ U[mu] @ np.conj(np.transpose(G[m], (0, 2, 1)))
    gpsi = np.einsum("nab,nsb->nsa", G, psi)
    lhs = O.apply(O.OP_MK, Ug, dims, gpsi, 0.12)
    rhs = np.einsum("nab,nsb->nsa", G, O.apply(O.OP_MK, U, dims, psi, 0.12))
    assert _rel(lhs, rhs) < 1e-14
    assert V == psi.shape[0]


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_gamma5_hermiticity_dense(dims):
    """M^dag = gamma5 M gamma5: the oracle's dagger is the conjugate transpose."""
    U = synth.gauge_field(dims, 0.5, seed=3)
    M = O.dense_operator(O.OP_MK, U, dims, 0.12)
    Md = O.dense_operator(O.OP_MK, U, dims, 0.12, dagger=True)
    assert np.allclose(Md, M.conj().T, atol=1e-15)
    g5 = np.kron(np.eye(synth.volume(dims)), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.allclose(g5 @ M @ g5, M.conj().T, atol=1e-15)


def test_paper_and_kappa_normalisations():
    """M_p(m) = (m + 4) M_k with kappa = 1/(2m + 8) (Eq. 3)."""
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 0.3, seed=1)
    psi = synth.gaussian_source(dims, seed=2)
    m = 0.3
    a = O.apply(O.OP_MP, U, dims, psi, m)
    b = (m + 4) * O.apply(O.OP_MK, U, dims, psi, O.kappa(m))
    assert _rel(a, b) < 1e-15


def test_L2_extent_accumulates_both_hops():
    """On an extent-2 direction n+mu = n-mu; both transporters must add.
    U = 1, constant spinor: each periodic direction gives psi[(1-g) + (1+g)] = 2 psi.
    Antiperiodic T = 2: at t = 0 the backward hop crosses the boundary, at t = 1
    the forward one, so the t terms give -2 psi g4 at t = 0 and +2 psi g4 at t = 1."""
    dims = (2, 2, 2, 2)
    g4 = O.gammas()[3]
    U = synth.unit_gauge_field(dims)
    psi = np.ones((16, 4, 3), dtype=np.complex128)
    out = O.hop(U, dims, psi, antiperiodic=False)
    assert np.allclose(out, 8.0 * psi, atol=0)
    out_ap = O.hop(U, dims, psi, antiperiodic=True)
    t = synth.lex_coords(dims)[:, 3]
    psig4 = np.einsum("nsc,st->ntc", psi, g4)
    want = 6.0 * psi + np.where(t == 0, -2.0, 2.0)[:, None, None] * psig4
    assert np.allclose(out_ap, want, atol=0)


# ------------------------------------------------------------------ solvers

def test_bicgstab_vs_dense_lu():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, seed=11)
    b = synth.gaussian_source(dims, seed=12)
    for m0 in (0.5, 0.1, -0.3):
        k = O.kappa(m0)
        x, st = O.bicgstab(O.OP_MK, U, dims, b, k, tol=1e-13)
        M = O.dense_operator(O.OP_MK, U, dims, k)
        xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
        assert st["status"] == O.OK
        assert _rel(x, xd) < 1e-12


def test_bicgstab_dagger_vs_dense_lu():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, seed=13)
    b = synth.gaussian_source(dims, seed=14)
    k = O.kappa(0.2)
    x, st = O.bicgstab(O.OP_MK, U, dims, b, k, tol=1e-13, dagger=True)
    M = O.dense_operator(O.OP_MK, U, dims, k)
    xd = np.linalg.solve(M.conj().T, b.reshape(-1)).reshape(b.shape)
    assert _rel(x, xd) < 1e-12


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_eo_solve_vs_dense_full_solve(dims):
    U = synth.gauge_field(dims, 0.5, seed=21)
    b = synth.z2_source(dims, seed=22)
    for m0 in (0.4, 0.05):
        x, st = O.eo_solve(U, dims, b, m0, tol=1e-12)
        M_full = O.dense_operator(O.OP_MK, U, dims, O.kappa(m0))
        xd = np.linalg.solve(M_full, b.reshape(-1)).reshape(b.shape)
        assert _rel(x, xd) < 1e-10
        assert st["true_relres_full"] < 1e-12


def test_mprec_is_schur_complement():
    """M_prec = 1 - kappa^2 D_eo D_oe is the even-even Schur complement of M_k."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, seed=5)
    k = 0.12
    M = O.dense_operator(O.OP_MK, U, dims, k)
    odd = np.repeat(O.parity_mask(dims), 12)
    Mee, Meo, Moe, Moo = M[~odd][:, ~odd], M[~odd][:, odd], M[odd][:, ~odd], M[odd][:, odd]
    S = Mee - Meo @ np.linalg.solve(Moo, Moe)
    P = O.dense_operator(O.OP_MPREC, U, dims, k)
    assert np.allclose(P[~odd][:, ~odd], S, atol=1e-14)
    assert np.allclose(P[odd], 0)


def test_bicgstab_m_vs_dense_lu():
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.5, seed=31)
    b = synth.z2_source(dims, seed=32)
    masses = [0.4, 0.25, 0.1, 0.05]
    xs, st = O.bicgstab_m(U, dims, b, masses, tol=1e-12)
    assert st["status"] == O.OK
    for m, x in zip(masses, xs):
        M = O.dense_operator(O.OP_MK, U, dims, O.kappa(m))
        xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
        assert _rel(x, xd) < 1e-9, m


def test_bicgstab_m_point_source_rhat_b_breaks_down():
    """With b a point source and the shadow residual rhat = b, rho_1 =
    <b, r_1> is exactly zero: r_1 at the source site is built from closed
    two-hop paths, all backtracks on extents >= 4, and (1 - gamma_mu)(1 +
    gamma_mu) = 0.  The recurrences must stop with a breakdown at once."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, seed=35)
    b = synth.point_source(dims)
    xs, st = O.bicgstab_m(U, dims, b, [0.4, 0.1], tol=1e-10, maxiter=50)
    assert st["status"] == O.BREAKDOWN and max(st["iterations"]) == 1, st
    # the same cancellation by hand: one BiCGstab step on M_p(0.1)
    A = lambda v: O.apply(O.OP_MP, U, dims, v, 0.1)
    v = A(b)
    s_ = b - (np.vdot(b, b) / np.vdot(b, v)) * v
    t = A(s_)
    r1 = s_ - (np.vdot(t, s_) / np.vdot(t, t)) * t
    assert abs(np.vdot(b, r1)) < 1e-16 * np.linalg.norm(r1)


def test_bicgstab_m_point_source_random_shadow_vs_dense_lu():
    """A Gaussian shadow residual removes the breakdown: every shifted
    solution of the point source matches dense LU."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, seed=36)
    b = synth.point_source(dims, 2, 1)
    rh = synth.gaussian_source(dims, seed=37)
    masses = [0.4, 0.2, 0.05]
    xs, st = O.bicgstab_m(U, dims, b, masses, tol=1e-12, rhat=rh)
    assert st["status"] == O.OK, st
    for m, x in zip(masses, xs):
        M = O.dense_operator(O.OP_MK, U, dims, O.kappa(m))
        xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
        assert _rel(x, xd) < 1e-9, m


def test_bicgstab_m_collinearity():
    """Truncated after k iterations, every shifted true residual is the
    unshifted residual divided by the scalar pi_k lambda_k: the residual
    vectors are collinear, |<r_s, r_i>| = ||r_s|| ||r_i||."""
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, seed=33)
    b = synth.gaussian_source(dims, seed=34)
    masses = [0.5, 0.3, 0.1]
    for k in (2, 5, 9):
        xs, st = O.bicgstab_m(U, dims, b, masses, tol=1e-30, maxiter=k)
        # r_i = b - M_p(m_i) psi_i  (psi_i = x_i / (m_i + 4))
        r = [b - O.apply(O.OP_MP, U, dims, x / (m + 4), m) for m, x in zip(masses, xs)]
        rs = r[2]  # unshifted (lightest mass)
        for ri in r[:2]:
            cosang = abs(np.vdot(rs, ri)) / (np.linalg.norm(rs) * np.linalg.norm(ri))
            assert abs(cosang - 1) < 1e-10


# -------------------------------------------------------- initial guesses

def test_lagrange_reproduces_polynomials():
    ms = [0.4, 0.35, 0.3, 0.25, 0.2]
    coeffs = [rng.standard_normal(24) for _ in range(len(ms))]
    poly = lambda m: sum(c * m ** j for j, c in enumerate(coeffs[:len(ms)]))
    for k in range(1, len(ms) + 1):
        # degree k-1 polynomial through k points is reproduced exactly
        pk = lambda m: sum(c * m ** j for j, c in enumerate(coeffs[:k]))
        w = O.lagrange_weights(ms[:k], 0.1)
        assert abs(w.sum() - 1) < 1e-12
        est = sum(wj * pk(mj) for wj, mj in zip(w, ms[:k]))
        assert np.allclose(est, pk(0.1), rtol=1e-10, atol=1e-10)
    assert poly(0.1).shape == (24,)


def test_ssm_is_least_squares_and_dk_identity():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, seed=41)
    b = synth.z2_source(dims, seed=42)
    prev = [0.5, 0.4, 0.3]
    psis = []
    for m in prev:
        x, _ = O.bicgstab(O.OP_MK, U, dims, b, O.kappa(m), tol=1e-13)
        psis.append(x / (m + 4))
    m = 0.2
    # d_k = b + (m - m_k) psi_k equals M_p(m) psi_k
    for mk, pk in zip(prev, psis):
        assert _rel(O.apply(O.OP_MP, U, dims, pk, m), b + (m - mk) * pk) < 1e-12
    c = O.ssm_coefficients(b, psis, prev, m)
    D = np.stack([(b + (m - mk) * pk).reshape(-1) for mk, pk in zip(prev, psis)], axis=1)
    c_ls = np.linalg.lstsq(D, b.reshape(-1), rcond=None)[0]
    assert np.allclose(c, c_ls, rtol=1e-8, atol=1e-10)


def test_initial_guesses_window_and_ssm_optimality():
    """Guesses from previous solutions: one previous solution extrapolates to
    psi_1 itself; two give the straight line through them; and the SSM
    guess has the smallest full residual of any combination in the span of
    the same solutions, so it beats the Lagrange guess from that span."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, seed=43)
    b = synth.z2_source(dims, seed=44)
    prev = [0.5, 0.4, 0.3]
    psis = [O.bicgstab(O.OP_MK, U, dims, b, O.kappa(mk), tol=1e-13)[0] / (mk + 4) for mk in prev]
    m = 0.2
    g1 = O.initial_guess(b, psis, prev, m, "poly", guess_max=1)
    assert _rel(g1, (m + 4) * psis[-1]) < 1e-15
    g2 = O.initial_guess(b, psis, prev, m, "poly", guess_max=2)
    line = psis[2] + (m - prev[2]) / (prev[1] - prev[2]) * (psis[1] - psis[2])
    assert _rel(g2, (m + 4) * line) < 1e-13
    res = lambda x: np.linalg.norm(b - O.apply(O.OP_MK, U, dims, x, O.kappa(m)))
    for k in (1, 2, 3):
        gs = O.initial_guess(b, psis, prev, m, "ssm", guess_max=k)
        gp = O.initial_guess(b, psis, prev, m, "poly", guess_max=k)
        assert res(gs) <= res(gp) * (1 + 1e-9), k
        # optimality: no perturbation within the span lowers the residual
        for pk in psis[-k:]:
            for eps in (1e-3, -1e-3, 1e-3j):
                assert res(gs) <= res(gs + eps * (m + 4) * pk) * (1 + 1e-12)
    assert O.initial_guess(b, psis, prev, m, "zero") is None


def test_multimass_scheme_converges():
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 0.3, seed=51)
    b = synth.point_source(dims)
    masses = [0.5, 0.3, 0.2, 0.1]
    xs, stats = O.multimass_solve(U, dims, b, masses, tol=1e-10)
    for m, x, st in zip(masses, xs, stats):
        assert O.true_relres(U, dims, b, x, m) < 1e-10
        M = O.dense_operator(O.OP_MK, U, dims, O.kappa(m))
        xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
        assert _rel(x, xd) < 1e-8


# ---------------------------------------------------------------- backward

def _su3_exp(h, coeffs):
    """exp(i h sum_a w_a lambda_a / 2) for coefficient arrays (..., 8)."""
    H = np.einsum("...a,aij->...ij", coeffs, synth.gell_mann() / 2.0)
    w, V = np.linalg.eigh(H)
    return np.einsum("...ik,...k,...jk->...ij", V, np.exp(1j * h * w), np.conj(V))


def _loss(U, dims, eta, masses):
    L = 0.0
    for m in masses:
        M = O.dense_operator(O.OP_MK, U, dims, O.kappa(m))
        x = np.linalg.solve(M, eta.reshape(-1))
        L += float(np.vdot(x, x).real)
    return L


def test_backward_vs_finite_differences():
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, seed=61)
    eta = synth.gaussian_source(dims, seed=62)
    masses = [0.4, 0.2]
    xs = []
    for m in masses:
        M = O.dense_operator(O.OP_MK, U, dims, O.kappa(m))
        xs.append(np.linalg.solve(M, eta.reshape(-1)).reshape(eta.shape))
    grads = [2.0 * x for x in xs]            # L = sum ||x||^2
    dU, dm = O.backward(U, dims, eta, masses, grads, xs=xs, tol=1e-14)
    h = 1e-5
    for trial in range(3):
        w = synth.su3_directions(dims, seed=100 + trial)
        Up = np.einsum("mnab,mnbc->mnac", _su3_exp(h, w), U)
        Um = np.einsum("mnab,mnbc->mnac", _su3_exp(-h, w), U)
        fd = (_loss(Up, dims, eta, masses) - _loss(Um, dims, eta, masses)) / (2 * h)
        an = float(np.sum(w * dU))
        assert abs(fd - an) / abs(an) < 1e-6, (fd, an)
    for i, m in enumerate(masses):
        hm = 1e-5
        fd = (_loss(U, dims, eta, [m + hm]) - _loss(U, dims, eta, [m - hm])) / (2 * hm)
        assert abs(fd - dm[i]) / abs(dm[i]) < 1e-6


def test_mass_gradient_free_field_closed_form():
    """Plane-wave source on U = 1: x_n = e^{ipn} c (u^T M(p)^{-1}), so
    L = V |c|^2 |u^T M(p)^{-1}|^2 and dL/dm0 follows from dM/dm0 = 2 kappa^2 D(p)."""
    dims = (4, 2, 2, 4)
    g = O.gammas()
    U = synth.unit_gauge_field(dims)
    u = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    eta, p, _ = _plane_wave(dims, [1, 1, 0, 2], c, u)
    m = 0.15
    k = O.kappa(m)
    Dp = _Dp(p, g)
    Mi = np.linalg.inv(np.eye(4) - k * Dp)
    w = u @ Mi
    dw = -u @ Mi @ (2 * k * k * Dp) @ Mi
    V = synth.volume(dims)
    want = V * np.vdot(c, c).real * 2 * np.vdot(w, dw).real
    x, _ = O.bicgstab(O.OP_MK, U, dims, eta, k, tol=1e-14)
    _, dm = O.backward(U, dims, eta, [m], [2 * x], xs=[x], tol=1e-14)
    assert abs(dm[0] - want) / abs(want) < 1e-9


def test_sampled_residual_helper_matches_full_residual():
    """The sampled-site residual used for the large lattices: over all sites
    its estimate is the full oracle residual, and the single-site peak never
    exceeds it."""
    from helpers import SampledResidual
    dims = (4, 4, 2, 6)
    U = synth.gauge_field(dims, 0.7, seed=5)
    b = synth.point_source(dims, 1, 2)
    m = 0.02
    x, _ = O.bicgstab(O.OP_MK, U, dims, b, O.kappa(m), tol=1e-6)
    full = O.true_relres(U, dims, b, x, m)
    est, peak = SampledResidual(dims, U, n_random=10 ** 6)(x, b, m)
    assert abs(est - full) <= 1e-12 * full
    est, peak = SampledResidual(dims, U, n_random=40)(x, b, m)
    assert peak <= full and 0.2 * full < est < 5 * full


def test_rightmost_eigenvalue_of_the_hop():
    """The critical-mass estimate's eigensolver (Krylov-Schur, largest real
    part) on the oracle's hop: equal to the dense spectrum's rightmost
    eigenvalue, and for U = 1 to the free-field edge 2 (3 + cos(pi/T))."""
    pytest.importorskip("scipy")
    import torch
    from paper_1103_5103_gb300.mass_sets import rightmost_eigenvalue
    for dims, U in (((4, 4, 4, 4), synth.gauge_field((4, 4, 4, 4), 0.5, seed=5)),
                    ((4, 4, 2, 6), synth.unit_gauge_field((4, 4, 2, 6)))):
        mv = lambda x: torch.from_numpy(O.hop(U, dims, x.numpy().reshape(-1, 4, 3)).reshape(-1))
        mu, ok, _ = rightmost_eigenvalue(mv, torch.from_numpy(synth.gaussian_source(dims, seed=11).reshape(-1)),
                                         tol=1e-12)
        assert ok
        dense = np.linalg.eigvals(O.dense_operator(O.OP_HOP, U, dims))
        assert abs(mu.real - dense.real.max()) < 1e-8
    assert abs(mu.real - 2 * (3 + np.cos(np.pi / 6))) < 1e-8
