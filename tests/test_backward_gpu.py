"""Backward of the multi-mass solve on the GPU: against the FP64 oracle's
gradient and against central finite differences (h = 1e-5) along random
su(3) directions, for L = sum_m ||x_m||^2 with x_m = M(m0)^{-1} eta."""
import numpy as np
import pytest
import torch

from helpers import rel
from oracle import oracle as O
from paper_1103_5103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1103_5103_gb300 import api, autograd
    return api, autograd


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _exp_su3(h, w):
    """exp(i h sum_a w_a lambda_a / 2) for coefficient arrays (..., 8)."""
    H = np.einsum("...a,aij->...ij", w, synth.gell_mann() / 2.0)
    ev, V = np.linalg.eigh(H)
    return np.einsum("...ik,...k,...jk->...ij", V, np.exp(1j * h * ev), np.conj(V))


def _loss(api, lat, U, eta, masses, prm):
    g = api.Gauge(lat, _cuda(U), precs=("f64", "f32", "df"))
    xs, st = api.multimass_solve(g, [_cuda(eta)], masses, prm)
    for s in st[0]:
        assert s["true_relres"] <= 2 * prm.tol, s
    return sum(float(torch.sum(torch.abs(x) ** 2)) for x in xs[0])


def test_backward_vs_oracle(mods):
    api, ag = mods
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.5, seed=71)
    eta = synth.gaussian_source(dims, seed=72)
    masses = [0.4, 0.2]
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U), precs=("f64", "f32", "df"))
    prm = api.params(tol=1e-12)
    xs, _ = api.multimass_solve(g, [_cuda(eta)], masses, prm)
    grads = [2.0 * x for x in xs[0]]
    dU, dm, db = api.solve_backward(g, _cuda(eta), grads, masses, xs=xs[0], prm=prm)
    xo = [O.bicgstab(O.OP_MK, U, dims, eta, O.kappa(m), tol=1e-13)[0] for m in masses]
    dU_o, dm_o = O.backward(U, dims, eta, masses, [2 * x for x in xo], xs=xo, tol=1e-13)
    assert rel(dU.cpu().numpy(), dU_o) < 1e-8
    assert np.allclose(dm, dm_o, rtol=1e-8, atol=0)
    # dL/d eta* = sum_m lam_m, lam_m = M^{-dag} g_m
    lam = sum(O.bicgstab(O.OP_MK, U, dims, 2 * x, O.kappa(m), tol=1e-13, dagger=True)[0] for x, m in zip(xo, masses))
    assert rel(db.cpu().numpy(), lam) < 1e-8


@pytest.mark.parametrize("dims,inner", [((8, 8, 8, 8), "f32"), ((8, 8, 8, 8), "f64")])
def test_autograd_vs_finite_differences(mods, dims, inner):
    """C4: L = sum over 4 masses of ||x_m||^2; 16 random su(3) directions,
    central differences with h = 1e-5, solves to 1e-13; bound 1e-6 relative."""
    api, ag = mods
    U = synth.gauge_field(dims, 0.3, seed=81)
    eta = synth.gaussian_source(dims, seed=82)
    masses = [0.5, 0.3, 0.2, 0.1]
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U), precs=("f64", "f32", "df"))
    prm = api.params(tol=1e-13, inner_prec=inner)
    eta_t = _cuda(eta).requires_grad_(True)
    m0 = torch.tensor(masses, dtype=torch.float64, device="cuda", requires_grad=True)
    omega = torch.zeros((4, lat.volume, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    x = ag.wilson_solve(g, eta_t, m0, omega, prm)
    L = torch.sum(torch.abs(x) ** 2)
    L.backward()
    dU = omega.grad.cpu().numpy()
    h = 1e-5
    worst = 0.0
    for k in range(16):
        w = synth.su3_directions(dims, seed=1000 + k)
        Up = np.einsum("mnab,mnbc->mnac", _exp_su3(h, w), U)
        Um = np.einsum("mnab,mnbc->mnac", _exp_su3(-h, w), U)
        fd = (_loss(api, lat, Up, eta, masses, prm) - _loss(api, lat, Um, eta, masses, prm)) / (2 * h)
        an = float(np.sum(w * dU))
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst < 1e-6, worst
    # masses
    gm = m0.grad.cpu().numpy()
    for i in range(len(masses)):
        mp, mm = list(masses), list(masses)
        mp[i] += h
        mm[i] -= h
        fd = (_loss(api, lat, U, eta, mp, prm) - _loss(api, lat, U, eta, mm, prm)) / (2 * h)
        assert abs(fd - gm[i]) / abs(gm[i]) < 1e-6, (i, fd, gm[i])
    # source: L is quadratic in eta, dL = Re <grad, d eta>
    d = synth.z2_source(dims, seed=83)
    fd = (_loss(api, lat, U, eta + h * d, masses, prm) - _loss(api, lat, U, eta - h * d, masses, prm)) / (2 * h)
    an = float(np.real(np.vdot(eta_t.grad.cpu().numpy(), d)))
    assert abs(fd - an) / abs(an) < 1e-6


def test_autograd_16x4_fp32_directions(mods):
    """C4 at 16^4 with an FP32 inner solve: four su(3) directions and one mass."""
    api, ag = mods
    dims = (16, 16, 16, 16)
    U = synth.gauge_field(dims, 0.3, seed=85)
    eta = synth.gaussian_source(dims, seed=86)
    masses = [0.5, 0.3, 0.2, 0.1]
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U), precs=("f64", "f32", "df"))
    prm = api.params(tol=1e-13, inner_prec="f32")
    m0 = torch.tensor(masses, dtype=torch.float64, device="cuda", requires_grad=True)
    omega = torch.zeros((4, lat.volume, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    x = ag.wilson_solve(g, _cuda(eta), m0, omega, prm, store_solutions=False)
    torch.sum(torch.abs(x) ** 2).backward()
    dU = omega.grad.cpu().numpy()
    h = 1e-5
    for k in range(4):
        w = synth.su3_directions(dims, seed=2000 + k)
        Up = np.einsum("mnab,mnbc->mnac", _exp_su3(h, w), U)
        Um = np.einsum("mnab,mnbc->mnac", _exp_su3(-h, w), U)
        fd = (_loss(api, lat, Up, eta, masses, prm) - _loss(api, lat, Um, eta, masses, prm)) / (2 * h)
        an = float(np.sum(w * dU))
        assert abs(fd - an) / abs(an) < 1e-6, (k, fd, an)
    mp = list(masses)
    mp[3] += h
    mm = list(masses)
    mm[3] -= h
    fd = (_loss(api, lat, U, eta, mp, prm) - _loss(api, lat, U, eta, mm, prm)) / (2 * h)
    assert abs(fd - m0.grad[3].item()) / abs(m0.grad[3].item()) < 1e-6


def test_backward_resolve_equals_stored(mods):
    api, ag = mods
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.3, seed=91)
    eta = synth.gaussian_source(dims, seed=92)
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(U), precs=("f64", "f32", "df"))
    prm = api.params(tol=1e-12)
    outs = []
    for store in (True, False):
        m0 = torch.tensor([0.3, 0.15], dtype=torch.float64, device="cuda", requires_grad=True)
        omega = torch.zeros((4, lat.volume, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        x = ag.wilson_solve(g, _cuda(eta), m0, omega, prm, store_solutions=store)
        torch.sum(torch.abs(x) ** 2).backward()
        outs.append((omega.grad.cpu().numpy(), m0.grad.cpu().numpy()))
    assert rel(outs[0][0], outs[1][0]) < 1e-9
    assert np.allclose(outs[0][1], outs[1][1], rtol=1e-9)


def test_backward_free_field_mass_derivative(mods):
    """Plane-wave source on U = 1: dL/dm0 has the closed form of the oracle pin."""
    api, ag = mods
    dims = (4, 4, 4, 8)
    g5 = O.gammas()
    U = synth.unit_gauge_field(dims)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    k = [1, 2, 0, 3]
    p = np.array([2 * np.pi * k[0] / 4, 2 * np.pi * k[1] / 4, 2 * np.pi * k[2] / 4, (2 * k[3] + 1) * np.pi / 8])
    phase = np.exp(1j * synth.lex_coords(dims) @ p)
    eta = phase[:, None, None] * np.einsum("s,c->sc", u, c)[None]
    m = 0.15
    kap = 1.0 / (2 * m + 8)
    Dp = sum(2 * np.cos(p[mu]) * np.eye(4) - 2j * np.sin(p[mu]) * g5[mu] for mu in range(4))
    Mi = np.linalg.inv(np.eye(4) - kap * Dp)
    w = u @ Mi
    dw = -u @ Mi @ (2 * kap * kap * Dp) @ Mi
    want = synth.volume(dims) * np.vdot(c, c).real * 2 * np.vdot(w, dw).real
    lat = api.Lattice(dims)
    gg = api.Gauge(lat, _cuda(U), precs=("f64", "f32", "df"))
    m0 = torch.tensor([m], dtype=torch.float64, device="cuda", requires_grad=True)
    x = ag.wilson_solve(gg, _cuda(eta), m0, None, api.params(tol=1e-13))
    torch.sum(torch.abs(x) ** 2).backward()
    assert abs(m0.grad.item() - want) / abs(want) < 1e-8
