"""The fused vector kernels of the BiCGstab iteration (Section 5's vector
utilities, one pass per update with its reductions), called directly
through wl_vector_op at half-lattice sizes that are not multiples of the
128-thread block (8, 24, 40 and 1080 sites: one partial block, and eight
full blocks plus a ragged ninth) and with 1, 3 and 7 right-hand sides:
every output element against numpy in FP64 on the stored inputs, every
reduction against math.fsum of the exact products, in FP64, FP32 and FP16
storage.  The solver tests see these kernels only through iteration counts;
a wrong last block of the grid reduction would show here."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1103_5103_gb300 import synth

pytestmark = pytest.mark.gpu

LATTICES = [(2, 2, 2, 2), (6, 2, 2, 2), (2, 2, 2, 10), (10, 6, 6, 6)]
# element tolerance relative to the largest reference element; reductions relative
ELEM = {"f64": 1e-14, "f32": 2e-6, "f16": 2e-3}
RED = {"f64": 1e-13, "f32": 1e-5, "f16": 1e-5}


@pytest.fixture(scope="module")
def api():
    from paper_1103_5103_gb300 import api as A
    return A


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class Vecs:
    """n_rhs internal even-site vectors of one precision in one buffer."""

    def __init__(self, lat, prec, stride, arrays):
        self.lat, self.prec, self.stride, self.n = lat, prec, stride, len(arrays)
        self.buf = torch.zeros(stride * self.n, dtype=torch.uint8, device="cuda")
        for r, a in enumerate(arrays):
            lat.spinor_import(_cuda(a), self.buf[r * stride:(r + 1) * stride], prec, 0)

    def values(self):
        """The stored values at the even sites, (n_rhs, Vh * 12) complex128."""
        even = ~O.parity_mask(self.lat.dims)
        out = []
        for r in range(self.n):
            full = torch.zeros((self.lat.volume, 4, 3), dtype=torch.complex128, device="cuda")
            self.lat.spinor_export(self.buf[r * self.stride:(r + 1) * self.stride], full, self.prec, 0)
            out.append(full.cpu().numpy()[even].reshape(-1))
        return np.array(out)


def _close(got, want, tol):
    scale = max(float(np.max(np.abs(want))), 1e-300)
    return float(np.max(np.abs(got - want))) <= tol * scale


def _fsum_dot(a, b):
    """sum conj(a) b in exact-rounding summation of the real and imaginary parts."""
    p = np.conj(a) * b
    return complex(math.fsum(p.real.tolist()), math.fsum(p.imag.tolist()))


def _setup(api, dims, prec, nrhs, nvec, seed):
    lat = api.Lattice(dims)
    g = api.Gauge(lat, _cuda(synth.unit_gauge_field(dims)), precs=(prec,))
    width = max(lat.spinor_bytes(prec), lat.spinor_bytes("f64" if prec == "f64" else "f32"))
    stride = (width + 255) // 256 * 256
    rng = np.random.default_rng(seed)
    arrays = [[synth.gaussian_source(dims, seed=int(rng.integers(1 << 30))) for _ in range(nrhs)]
              for _ in range(nvec)]
    scal = [(complex(*rng.normal(size=2)), complex(*rng.normal(size=2)), complex(*rng.normal(size=2)))
            for _ in range(nrhs)]
    return lat, g, stride, arrays, scal


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("nrhs", [1, 3, 7])
@pytest.mark.parametrize("dims", LATTICES)
def test_s_and_p_updates(api, dims, nrhs, prec):
    lat, g, stride, arrays, scal = _setup(api, dims, prec, nrhs, 3, 11)
    r, v, s = (Vecs(lat, prec, stride, a) for a in arrays)
    R, Vv = r.values(), v.values()
    api.vector_op(g, api.VEC_S, prec, nrhs, stride, [r.buf, v.buf, s.buf], scal)
    al = np.array([c[0] for c in scal])[:, None]
    assert _close(s.values(), R - al * Vv, ELEM[prec])
    p = Vecs(lat, prec, stride, arrays[2])
    P = p.values()
    api.vector_op(g, api.VEC_P, prec, nrhs, stride, [r.buf, p.buf, v.buf], scal)
    om = np.array([c[1] for c in scal])[:, None]
    be = np.array([c[2] for c in scal])[:, None]
    assert _close(p.values(), R + be * (P - om * Vv), ELEM[prec])


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("nrhs", [1, 3, 7])
@pytest.mark.parametrize("dims", LATTICES)
def test_xr_update_and_its_reductions(api, dims, nrhs, prec):
    """x += alpha p + omega s and r = s - omega t, with <rhat, r> and
    ||r||^2 of the new r reduced over the grid (the scalars beta and rho
    of the next iteration come from them)."""
    lat, g, stride, arrays, scal = _setup(api, dims, prec, nrhs, 6, 12)
    xprec = "f64" if prec == "f64" else "f32"
    x = Vecs(lat, xprec, stride, arrays[0])
    p, s, t, r, rh = (Vecs(lat, prec, stride, a) for a in arrays[1:])
    X, P, S, T, RH = x.values(), p.values(), s.values(), t.values(), rh.values()
    dots = api.vector_op(g, api.VEC_XR, prec, nrhs, stride, [x.buf, p.buf, s.buf, t.buf, r.buf, rh.buf], scal)
    al = np.array([c[0] for c in scal])[:, None]
    om = np.array([c[1] for c in scal])[:, None]
    assert _close(x.values(), X + al * P + om * S, ELEM[xprec])
    Rn = r.values()
    assert _close(Rn, S - om * T, ELEM[prec])
    for k in range(nrhs):
        d = _fsum_dot(RH[k], Rn[k])
        n2 = math.fsum((np.abs(Rn[k]) ** 2).tolist())
        got = complex(dots[3 * k], dots[3 * k + 1])
        assert abs(got - d) <= RED[prec] * math.sqrt(n2 * math.fsum((np.abs(RH[k]) ** 2).tolist())), (k, got, d)
        assert abs(dots[3 * k + 2] - n2) <= RED[prec] * n2, (k, dots[3 * k + 2], n2)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("nrhs", [1, 3, 7])
@pytest.mark.parametrize("dims", LATTICES)
def test_norm2(api, dims, nrhs, prec):
    lat, g, stride, arrays, _ = _setup(api, dims, prec, nrhs, 1, 13)
    a = Vecs(lat, prec, stride, arrays[0])
    A = a.values()
    got = api.vector_op(g, api.VEC_NORM2, prec, nrhs, stride, [a.buf])
    for k in range(nrhs):
        want = math.fsum((np.abs(A[k]) ** 2).tolist())
        assert abs(got[k] - want) <= RED[prec] * want, (k, got[k], want)
