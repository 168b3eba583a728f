"""FP64 CPU oracle for the Wilson multi-mass solve (arXiv:1103.5103).

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA path is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it.  The library never calls it and
the two share no code; the only common inputs are the seeded fields from
``paper_1103_5103_gb300.synth``, which callers generate and pass in.

The hop, the operators, BiCGstab, BiCGstab-M and the link force are plain C
(``wilson_oracle.c``); this module wraps them and adds the numpy steps of the
paper's single-mass scheme: even-odd preconditioning (Section 6.2.3), the
Lagrange initial guess (Section 6.2.1, Eq. Poly and the closed-form
Vandermonde solution), the solution-space-minimisation guess (Section 6.2.2)
and the adjoint-solve backward.

Vectors are canonical complex128 arrays of shape (V, 4, 3) (spin, colour),
links (4, V, 3, 3).  Everything is FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OP_HOP, OP_MK, OP_MP, OP_MPREC = 0, 1, 2, 3
OK, NOCONV = 0, 1


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, no contraction so x86 and Arm agree),
    with OpenMP for the per-site loops where the compiler has it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fcx-limited-range",
                "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int = 0) -> int:
    """Threads for the oracle's per-site loops (n > 0 sets them); returns the
    count in use.  Results do not depend on it."""
    return int(lib().or_threads(int(n)))


class _Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dims", ctypes.c_int * 4), ("antiperiodic_t", ctypes.c_int),
                ("dagger", ctypes.c_int), ("param", ctypes.c_double), ("U", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_relres", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        _lib.or_hop.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        _lib.or_gamma5.argtypes = [vp, vp, vp]
        _lib.or_apply.argtypes = [ctypes.POINTER(_Op), vp, vp]
        _lib.or_bicgstab.argtypes = [ctypes.POINTER(_Op), vp, vp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.POINTER(_Stats)]
        _lib.or_bicgstab.restype = ctypes.c_int
        _lib.or_bicgstab_m.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp, vp,
                                       ctypes.c_double, ctypes.c_int, vp]
        _lib.or_bicgstab_m.restype = ctypes.c_int
        _lib.or_link_force.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_double, vp, vp]
        _lib.or_gamma_matrices.argtypes = [vp]
        _lib.or_apply_mk_sites.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, vp, ctypes.c_long, vp]
        _lib.or_threads.argtypes = [ctypes.c_int]
        _lib.or_threads.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def volume(dims) -> int:
    return int(np.prod(dims))


def kappa(m0: float) -> float:
    """kappa = 1 / (2 m0 + 8), so that M_p(m0) = (m0 + 4) M_k."""
    return 1.0 / (2.0 * m0 + 8.0)


def gammas() -> np.ndarray:
    """gamma_1..gamma_4 and gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4, shape (5, 4, 4)."""
    g = np.zeros((5, 4, 4), dtype=np.complex128)
    lib().or_gamma_matrices(_p(g))
    return g


def parity_mask(dims) -> np.ndarray:
    """Boolean (V,) array, True on odd sites."""
    X, Y, Z, T = dims
    n = np.arange(volume(dims))
    return ((n % X + (n // X) % Y + (n // (X * Y)) % Z + n // (X * Y * Z)) % 2) == 1


def hop(U, dims, psi, antiperiodic=True):
    """D psi over the whole lattice (Eq. 4 summed over mu = +-1..+-4)."""
    U, psi = _c128(U), _c128(psi)
    out = np.empty_like(psi)
    lib().or_hop(_dims(dims), int(antiperiodic), _p(U), _p(psi), _p(out))
    return out


def gamma5(dims, psi):
    psi = _c128(psi)
    out = np.empty_like(psi)
    lib().or_gamma5(_dims(dims), _p(psi), _p(out))
    return out


def _op(kind, dims, U, param=0.0, antiperiodic=True, dagger=False):
    op = _Op()
    op.kind = kind
    op.dims = _dims(dims)
    op.antiperiodic_t = int(antiperiodic)
    op.dagger = int(dagger)
    op.param = float(param)
    op.U = U.ctypes.data
    return op


def apply(kind, U, dims, psi, param=0.0, antiperiodic=True, dagger=False):
    """Apply HOP (D), MK (1 - kappa D), MP ((m+4) - D/2) or MPREC (1 - kappa^2 D_eo D_oe)."""
    U, psi = _c128(U), _c128(psi)
    out = np.empty_like(psi)
    op = _op(kind, dims, U, param, antiperiodic, dagger)
    lib().or_apply(ctypes.byref(op), _p(psi), _p(out))
    return out


def bicgstab(kind, U, dims, b, param, x0=None, tol=1e-10, bref=None, maxiter=10000,
             antiperiodic=True, dagger=False):
    """Solve A x = b with BiCGstab to ||b - A x|| <= tol * bref (bref defaults to ||b||)."""
    U, b = _c128(U), _c128(b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    if bref is None:
        bref = float(np.linalg.norm(b))
    st = _Stats()
    op = _op(kind, dims, U, param, antiperiodic, dagger)
    status = lib().or_bicgstab(ctypes.byref(op), _p(b), _p(x), tol, bref, maxiter, ctypes.byref(st))
    return x, dict(status=status, iterations=st.iterations, matvecs=st.matvecs,
                   restarts=st.restarts, true_relres=st.true_relres)


BREAKDOWN = 2


def bicgstab_m(U, dims, b, masses, tol=1e-10, maxiter=10000, antiperiodic=True, rhat=None):
    """BiCGstab-M on M_p(m_s) + sigma_i; returns kappa-form solutions x_i = (m_i+4) psi_i.
    rhat is the shadow residual (default b); status BREAKDOWN when <rhat, v>
    or rho vanishes, as it does after one iteration for a point source b
    with rhat = b."""
    U, b = _c128(U), _c128(b)
    rh = None if rhat is None else _c128(rhat)
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    outs = [np.zeros_like(b) for _ in masses]
    ptrs = (ctypes.c_void_p * len(masses))(*[o.ctypes.data for o in outs])
    iters = np.zeros(len(masses), dtype=np.int32)
    status = lib().or_bicgstab_m(_dims(dims), int(antiperiodic), _p(U), _p(masses), len(masses), _p(b),
                                 None if rh is None else _p(rh), ptrs, tol, maxiter, _p(iters))
    xs = [(m + 4.0) * o for m, o in zip(masses, outs)]
    return xs, dict(status=status, iterations=[int(i) for i in iters])


def apply_mk_sites(U, dims, psi, kappa, sites, antiperiodic=True):
    """(M_k psi)_n at the given lexicographic sites, shape (len(sites), 4, 3)."""
    U, psi = _c128(U), _c128(psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    lib().or_apply_mk_sites(_dims(dims), int(antiperiodic), _p(U), _p(psi), float(kappa), _p(sites), len(sites),
                            _p(out))
    return out


def true_relres(U, dims, b, x, m0, antiperiodic=True):
    """||b - M_k(m0) x|| / ||b|| on the full lattice."""
    r = b - apply(OP_MK, U, dims, x, kappa(m0), antiperiodic)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


# ------------------------------------------------------------- even-odd --

def eo_source(U, dims, b, m0, antiperiodic=True):
    """b_prec = b_e + kappa D_eo b_o (kappa form of Eq. eo4); odd sites zero."""
    odd = parity_mask(dims)
    bo = _c128(b).copy()
    bo[~odd] = 0
    Db = hop(U, dims, bo, antiperiodic)
    bp = _c128(b).copy() + kappa(m0) * Db
    bp[odd] = 0
    return bp


def eo_reconstruct(U, dims, b, xe, m0, antiperiodic=True):
    """x_o = b_o + kappa D_oe x_e (kappa form of Eq. eo3); returns the full x."""
    odd = parity_mask(dims)
    xe = _c128(xe).copy()
    xe[odd] = 0
    Dx = hop(U, dims, xe, antiperiodic)
    x = xe.copy()
    x[odd] = b[odd] + kappa(m0) * Dx[odd]
    return x


def eo_solve(U, dims, b, m0, x0e=None, tol=1e-10, maxiter=10000, antiperiodic=True):
    """Solve M_k(m0) x = b through M_prec x_e = b_prec, then reconstruct x_o.
    The inner stop uses ||r_prec|| <= tol ||b|| (the even part of the full
    residual equals the preconditioned residual when x_o is reconstructed)."""
    bp = eo_source(U, dims, b, m0, antiperiodic)
    xe, st = bicgstab(OP_MPREC, U, dims, bp, kappa(m0), x0=x0e, tol=tol,
                      bref=float(np.linalg.norm(b)), maxiter=maxiter, antiperiodic=antiperiodic)
    x = eo_reconstruct(U, dims, b, xe, m0, antiperiodic)
    st["true_relres_full"] = true_relres(U, dims, b, x, m0, antiperiodic)
    return x, st


# ------------------------------------------------------- initial guesses --

def lagrange_weights(m_prev, m):
    """w_j = prod_{i != j} (m - m_i) / (m_j - m_i): the closed-form solution of
    the Vandermonde system of Eq. Poly, evaluated at m (Section 6.2.1)."""
    m_prev = [float(v) for v in m_prev]
    w = []
    for j, mj in enumerate(m_prev):
        t = 1.0
        for i, mi in enumerate(m_prev):
            if i != j:
                t *= (m - mi) / (mj - mi)
        w.append(t)
    return np.array(w)


def ssm_coefficients(b, psis, m_prev, m):
    """Solution-space minimisation (Section 6.2.2): c solving
    sum_j c_j d_i^dag d_j = d_i^dag b with d_k = b + (m - m_k) psi_k,
    psi_k in the paper's normalisation."""
    d = [b.reshape(-1) + (m - mk) * pk.reshape(-1) for pk, mk in zip(psis, m_prev)]
    G = np.array([[np.vdot(di, dj) for dj in d] for di in d])
    rhs = np.array([np.vdot(di, b.reshape(-1)) for di in d])
    return np.linalg.solve(G, rhs)


def initial_guess(b, done_psi, done_m, m, guess="poly", guess_max=0):
    """Full-lattice kappa-form initial guess for mass m from the previous
    paper-normalised solutions psi_j (in solve order): Lagrange extrapolation
    (Section 6.2.1) or solution-space minimisation (Section 6.2.2) through the
    last guess_max of them (0: all).  None when there is nothing to use."""
    if guess == "zero" or not done_m:
        return None
    k = len(done_m) if guess_max <= 0 else min(guess_max, len(done_m))
    ms, ps = done_m[-k:], done_psi[-k:]
    if guess == "poly":
        c = lagrange_weights(ms, m)
    elif guess == "ssm":
        c = ssm_coefficients(b, ps, ms, m)
    else:
        raise ValueError(guess)
    return (m + 4.0) * sum(cj * pj for cj, pj in zip(c, ps))


def multimass_solve(U, dims, b, masses, tol=1e-10, guess="poly", maxiter=10000, antiperiodic=True, guess_max=0,
                    on_solution=None):
    """The paper's single-mass scheme (Section 6.2, Section 7): masses solved
    heaviest first, each by even-odd-preconditioned BiCGstab started from the
    polynomial extrapolation through all previous solutions (extrapolating the
    paper-normalised solution psi = x / (m + 4) on even sites), or from the
    solution-space minimisation guess.  Returns kappa-form solutions in the
    caller's mass order and per-mass stats.

    With on_solution, each solution is handed to on_solution(i, x, stats) as
    soon as it is found and is not kept (the returned xs[i] is None); the
    polynomial guess then stores only the even sites of the earlier psi, the
    only sites it uses, so that lattices of 10^7 sites fit in host memory.
    The arithmetic is the same either way."""
    order = sorted(range(len(masses)), key=lambda i: -masses[i])
    odd = parity_mask(dims)
    even = ~odd
    lean = on_solution is not None and guess == "poly"
    done_m, done_psi = [], []
    xs, stats = [None] * len(masses), [None] * len(masses)
    for i in order:
        m = float(masses[i])
        x0 = initial_guess(b, done_psi, done_m, m, guess, guess_max)
        if x0 is not None:
            if lean:
                full = np.zeros(np.shape(b), dtype=np.complex128)
                full[even] = x0
                x0 = full
            else:
                x0 = x0.copy()
                x0[odd] = 0
        x, st = eo_solve(U, dims, b, m, x0e=x0, tol=tol, maxiter=maxiter, antiperiodic=antiperiodic)
        del x0
        stats[i] = st
        done_m.append(m)
        done_psi.append((x[even] if lean else x) / (m + 4.0))
        if on_solution is None:
            xs[i] = x
        else:
            on_solution(i, x, st)
        del x
    return xs, stats


# -------------------------------------------------------------- backward --

def link_force(U, dims, x, lam, coef, antiperiodic=True):
    """-coef * Im tr(T_a W_mu(n)) per link and generator, shape (4, V, 8)."""
    from_gm = _gell_mann()
    U, x, lam = _c128(U), _c128(x), _c128(lam)
    force = np.zeros((4, volume(dims), 8), dtype=np.float64)
    lib().or_link_force(_dims(dims), int(antiperiodic), _p(U), _p(x), _p(lam), float(coef),
                        _p(from_gm), _p(force))
    return force


def _gell_mann():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def backward(U, dims, b, masses, grads, xs=None, tol=1e-12, antiperiodic=True):
    """Gradient of a real loss L(x_1..x_k), x_i = M_k(m_i)^{-1} b, given
    g_i = dL/dRe x_i + i dL/dIm x_i.  Solves the adjoint systems
    M_k^dag lam_i = g_i (through M^dag = gamma5 M gamma5) and returns
    (dL/dU as su(3) components (4, V, 8), dL/dm0 per mass) with
    dL/dm0 = -Re<lam, (dM/dm0) x> = -Re<lam, 2 kappa^2 D x>."""
    dU = np.zeros((4, volume(dims), 8))
    dm = np.zeros(len(masses))
    for i, m in enumerate(masses):
        k = kappa(m)
        x = xs[i] if xs is not None else bicgstab(OP_MK, U, dims, b, k, tol=tol, antiperiodic=antiperiodic)[0]
        lam, _ = bicgstab(OP_MK, U, dims, grads[i], k, tol=tol, dagger=True, antiperiodic=antiperiodic)
        dU += link_force(U, dims, x, lam, k, antiperiodic)
        Dx = hop(U, dims, x, antiperiodic)
        dm[i] = -np.real(np.vdot(lam, 2.0 * k * k * Dx))
    return dU, dm


# ------------------------------------------------------------ dense aids --

def dense_operator(kind, U, dims, param=0.0, antiperiodic=True, dagger=False, sites=None):
    """Dense matrix of an operator, assembled column by column (tiny lattices only)."""
    V = volume(dims)
    n = 12 * V
    cols = range(n) if sites is None else [12 * s + k for s in sites for k in range(12)]
    A = np.zeros((n, len(cols)), dtype=np.complex128)
    e = np.zeros((V, 4, 3), dtype=np.complex128)
    flat = e.reshape(-1)
    for j, c in enumerate(cols):
        flat[c] = 1.0
        A[:, j] = apply(kind, U, dims, e, param, antiperiodic, dagger).reshape(-1)
        flat[c] = 0.0
    return A
