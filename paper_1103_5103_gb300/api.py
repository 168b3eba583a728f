"""Thin ctypes binding of libwilson.so (the C ABI declared in include/wilson.h).

Argument marshalling only: every step of every call runs in the library's
sm_103a kernels.  PyTorch supplies device memory and the current stream.
The binding raises at import if the compiled library is missing -- there is
no CPU fallback.

Vectors are complex128 CUDA tensors in the canonical layout: spinors
(V, 4, 3) = [site][spin][colour], links (4, V, 3, 3) = [mu][site][row][col],
site n = x + X*(y + Y*(z + Z*t)).
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# WL_LIBRARY=checked loads the bounds-checked build (every internal site
# index tested, violations recorded instead of trapping)
LIB_PATH = os.path.join(_HERE, "libwilson_checked.so" if os.environ.get("WL_LIBRARY") == "checked"
                        else "libwilson.so")

WL_OK, WL_ERR_ARG, WL_ERR_CUDA, WL_ERR_OOM, WL_ERR_NOCONV, WL_ERR_BREAKDOWN, WL_ERR_TIMEOUT, WL_ERR_CHECKED = range(8)
F64, F32, F16, DF = 1, 2, 4, 8
EVEN, ODD = 0, 1
OP_HOP, OP_M, OP_MPREC = 0, 1, 2
GUESS_ZERO, GUESS_POLY, GUESS_SSM = 0, 1, 2
SOLVER_BICGSTAB, SOLVER_CG = 0, 1
MODE_HOST, MODE_GRAPH, MODE_PERSISTENT = 0, 1, 2
_PREC_NAMES = {"f64": F64, "f32": F32, "f16": F16, "df": DF}


def _prec(p) -> int:
    """'f64' | 'f32' | 'f16' | 'df' or the raw WL_F* value (validated by the library)."""
    return _PREC_NAMES[p] if isinstance(p, str) else int(p)


class WilsonError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libwilson status {status}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)
_vp, _int, _dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", _dbl), ("max_iter", _int), ("inner_prec", _int), ("inner_tol", _dbl),
                ("max_restarts", _int), ("guess", _int), ("mode", _int), ("rhs_block", _int),
                ("graph_iters", _int), ("eo", _int), ("outer_prec", _int), ("shadow", _vp),
                ("guess_max", _int), ("reliable", _int), ("inner_solver", _int), ("verify_full", _int),
                ("outer_blocks_per_sm", _int), ("inner_refine", _int)]


class SolverStats(ctypes.Structure):
    _fields_ = [("mass", _dbl), ("status", _int), ("iterations", _int), ("matvecs", _int),
                ("restarts", _int), ("true_relres", _dbl), ("seconds", _dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", _dbl), ("site_rhs", _dbl), ("sites", _dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _sig(name, args, res=_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("wl_last_error", [], ctypes.c_char_p)
_sig("wl_params_default", [ctypes.POINTER(SolverParams)])
_sig("wl_lattice_create", [ctypes.POINTER(_int), _int, ctypes.POINTER(_vp)])
_sig("wl_lattice_destroy", [_vp])
_sig("wl_spinor_bytes", [_vp, _int, ctypes.POINTER(ctypes.c_size_t)])
_sig("wl_spinor_import", [_vp, _vp, _vp, _int, _int, _vp])
_sig("wl_spinor_export", [_vp, _vp, _vp, _int, _int, _vp])
_sig("wl_gauge_create", [_vp, _vp, ctypes.c_uint, _vp, ctypes.POINTER(_vp)])
_sig("wl_gauge_destroy", [_vp])
_sig("wilson_hop", [_vp, _vp, _vp, _vp, _dbl, _int, _int, _int, _vp])
_sig("wilson_hop_multi", [_vp, _vp, _vp, _vp, _dbl, _int, _int, _int, _int, ctypes.c_size_t, _int, _vp])
_sig("wilson_dslash", [_vp, _vp, _vp, _dbl, _int, _int, _vp])
_sig("wilson_dslash_noalloc", [_vp, _vp, _vp, _dbl, _int, _int, _int, _vp])
_sig("wilson_dslash_dag", [_vp, _vp, _vp, _dbl, _int, _int, _vp])
_sig("bicgstab_solve", [_vp, _vp, _vp, _dbl, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), _vp])
_sig("wl_launch_count", [ctypes.POINTER(ctypes.c_longlong)])
_sig("wl_autotune", [_vp, _int, _int, _vp, ctypes.POINTER(_int), ctypes.POINTER(_dbl)])
_sig("wl_profile_enable", [_vp, _int])
_sig("wl_wait_faults", [ctypes.POINTER(ctypes.c_uint), _int, _vp])
_sig("wl_checked_status", [ctypes.POINTER(ctypes.c_ulonglong), _int])
_sig("wl_vector_op", [_vp, _int, _int, _int, ctypes.c_size_t, ctypes.POINTER(_vp), ctypes.POINTER(_dbl),
                      ctypes.POINTER(_dbl), _vp])
_sig("wl_is_checked_build", [])
_sig("wl_persistent_selftest", [_vp, _int, _int, _dbl, _vp])
_sig("wl_profile_read", [_vp, ctypes.POINTER(KernelProfile)])
_sig("wilson_solve_backward", [_vp, _vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(_dbl), _int,
                               ctypes.POINTER(SolverParams), _vp, ctypes.POINTER(_dbl), _vp, _vp])
_sig("bicgstab_m_solve", [_vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(_dbl), _int, ctypes.POINTER(SolverParams),
                          ctypes.POINTER(SolverStats), _vp])
_sig("multimass_solve", [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _int, ctypes.POINTER(_dbl), _int,
                         ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), _vp])


def lib():
    return _lib


def last_error() -> str:
    return (_lib.wl_last_error() or b"").decode()


def _check(status: int, allow=(WL_OK,)):
    if status not in allow:
        raise WilsonError(status, last_error())
    return status


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _canon(t: torch.Tensor, V: int, what: str):
    """Canonical source or solution: a CUDA tensor, or a page-locked host
    tensor that the kernels access directly (unified addressing)."""
    if t.dtype != torch.complex128 or t.numel() != 12 * V:
        raise ValueError(f"{what}: expected complex128 with {12 * V} entries (V, 4, 3)")
    if not t.is_cuda:
        if not t.is_pinned():
            raise ValueError(f"{what}: expected a CUDA tensor or pinned host memory")
        if not t.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous tensor")
        return ctypes.c_void_p(t.data_ptr())
    return _ptr(t)


def params(**kw) -> SolverParams:
    """Default solver parameters (wl_params_default) with keyword overrides;
    inner_prec accepts 'f64' | 'f32' | 'f16', outer_prec 'f64' | 'df' (the
    defect correction's outer loop, and the vectors and hops of
    bicgstab_m_solve); shadow takes a canonical complex128 CUDA tensor (kept
    alive by the returned object)."""
    p = SolverParams()
    _check(_lib.wl_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k in ("inner_prec", "outer_prec"):
            v = _prec(v)
        if k == "shadow" and v is not None:
            if v.dtype != torch.complex128:
                raise ValueError("shadow: expected a complex128 tensor")
            p._shadow = v
            v = _ptr(v).value
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Lattice:
    """wl_lattice handle: extents (X, Y, Z, T), all even."""

    def __init__(self, dims, antiperiodic_t: bool = True):
        self.dims = tuple(int(d) for d in dims)
        self.volume = 1
        for d in self.dims:
            self.volume *= d
        h = _vp()
        arr = (_int * 4)(*self.dims)
        _check(_lib.wl_lattice_create(arr, int(antiperiodic_t), ctypes.byref(h)))
        self.handle = h
        self.antiperiodic_t = bool(antiperiodic_t)

    def spinor_bytes(self, prec) -> int:
        n = ctypes.c_size_t()
        _check(_lib.wl_spinor_bytes(self.handle, _prec(prec), ctypes.byref(n)))
        return n.value

    def new_internal(self, prec, device="cuda") -> torch.Tensor:
        """Uninitialised internal (one-parity) spinor buffer."""
        return torch.empty(self.spinor_bytes(prec), dtype=torch.uint8, device=device)

    def spinor_import(self, canon: torch.Tensor, internal: torch.Tensor, prec, parity, stream=None):
        _check(_lib.wl_spinor_import(self.handle, _canon(canon, self.volume, "canon"), _ptr(internal), _prec(prec),
                                     parity, _stream(stream)))

    def spinor_export(self, internal: torch.Tensor, canon: torch.Tensor, prec, parity, stream=None):
        _check(_lib.wl_spinor_export(self.handle, _ptr(internal), _canon(canon, self.volume, "canon"), _prec(prec),
                                     parity, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            _lib.wl_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Gauge:
    """wl_gauge handle built from canonical complex128 CUDA links (4, V, 3, 3)."""

    def __init__(self, lat: Lattice, U: torch.Tensor, precs=("f64", "f32", "f16", "df"), stream=None):
        if U.dtype != torch.complex128 or U.numel() != 36 * lat.volume:
            raise ValueError("links: expected complex128 (4, V, 3, 3)")
        mask = 0
        for p in precs:
            mask |= _prec(p)
        h = _vp()
        _check(_lib.wl_gauge_create(lat.handle, _ptr(U), mask, _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.lat = lat

    def close(self):
        if getattr(self, "handle", None):
            _lib.wl_gauge_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wilson_hop(g: Gauge, inp: torch.Tensor, out: torch.Tensor, x, coef: float, prec, out_parity: int,
               dagger: bool = False, stream=None):
    """out = x + coef * D_{p,1-p} inp on internal spinors (x may be None)."""
    _check(_lib.wilson_hop(g.handle, _ptr(inp), _ptr(out), None if x is None else _ptr(x), float(coef), _prec(prec),
                           int(out_parity), int(dagger), _stream(stream)))


def hop_batch(g: Gauge, inp: torch.Tensor, out: torch.Tensor, nrhs: int, rhs_stride: int, coef: float, prec,
              out_parity: int, rhs_block: int = 1, x=None, dagger: bool = False, stream=None):
    """wilson_hop_multi: out_r = x_r + coef D in_r for nrhs internal spinors rhs_stride bytes apart."""
    _check(_lib.wilson_hop_multi(g.handle, _ptr(inp), _ptr(out), None if x is None else _ptr(x), float(coef),
                                 _prec(prec), int(out_parity), int(dagger), int(nrhs), int(rhs_stride),
                                 int(rhs_block), _stream(stream)))


def wilson_dslash(g: Gauge, inp: torch.Tensor, out: torch.Tensor, kappa: float, prec, op=OP_M, stream=None):
    V = g.lat.volume
    _check(_lib.wilson_dslash(g.handle, _canon(inp, V, "in"), _canon(out, V, "out"), float(kappa), _prec(prec),
                              int(op), _stream(stream)))


def wilson_dslash_dag(g: Gauge, inp: torch.Tensor, out: torch.Tensor, kappa: float, prec, op=OP_M, stream=None):
    V = g.lat.volume
    _check(_lib.wilson_dslash_dag(g.handle, _canon(inp, V, "in"), _canon(out, V, "out"), float(kappa), _prec(prec),
                                  int(op), _stream(stream)))


def wilson_dslash_noalloc(g: Gauge, inp: torch.Tensor, out: torch.Tensor, kappa: float, prec, op=OP_M,
                          dagger: bool = False, stream=None):
    """wilson_dslash without any device allocation (fixed 64 MiB scratch in the library)."""
    V = g.lat.volume
    _check(_lib.wilson_dslash_noalloc(g.handle, _canon(inp, V, "in"), _canon(out, V, "out"), float(kappa),
                                      _prec(prec), int(op), int(dagger), _stream(stream)))


def bicgstab_solve(g: Gauge, b: torch.Tensor, x: torch.Tensor, m0: float, prm: SolverParams | None = None,
                   stream=None, check=True) -> dict:
    """Solve M_k(m0) x = b (x: guess in, solution out).  Returns the stats dict."""
    prm = prm or params()
    st = SolverStats()
    V = g.lat.volume
    s = _lib.bicgstab_solve(g.handle, _canon(b, V, "b"), _canon(x, V, "x"), float(m0), ctypes.byref(prm),
                            ctypes.byref(st), _stream(stream))
    if check:
        _check(s)
    d = st.as_dict()
    d["call_status"] = s
    return d


def multimass_solve(g: Gauge, bs, masses, prm: SolverParams | None = None, xs=None, stream=None, check=True):
    """The paper's single-mass multi-mass scheme for every source in bs.
    Returns (xs, stats) with xs[r][i] the solution for source r, mass i."""
    prm = prm or params()
    V = g.lat.volume
    nr, nm = len(bs), len(masses)
    if xs is None:
        xs = [[torch.empty_like(b) if b.is_cuda else torch.empty_like(b).pin_memory() for _ in masses] for b in bs]
    bp = (_vp * nr)(*[_canon(b, V, "b").value for b in bs])
    xp = (_vp * (nr * nm))(*[_canon(xs[r][i], V, "x").value for r in range(nr) for i in range(nm)])
    ms = (_dbl * nm)(*[float(m) for m in masses])
    st = (SolverStats * (nr * nm))()
    s = _lib.multimass_solve(g.handle, bp, xp, nr, ms, nm, ctypes.byref(prm), st, _stream(stream))
    if check:
        _check(s)
    stats = [[st[r * nm + i].as_dict() for i in range(nm)] for r in range(nr)]
    return xs, stats


def bicgstab_m_solve(g: Gauge, b: torch.Tensor, xs, masses, prm: SolverParams | None = None, stream=None,
                     check=True):
    """Multi-shift BiCGstab-M baseline; xs[i] (canonical complex128) receives
    the solution for masses[i].  Returns per-mass stats dicts."""
    prm = prm or params()
    V = g.lat.volume
    nm = len(masses)
    xp = (_vp * nm)(*[_canon(x, V, "x").value for x in xs])
    ms = (_dbl * nm)(*[float(m) for m in masses])
    st = (SolverStats * nm)()
    s = _lib.bicgstab_m_solve(g.handle, _canon(b, V, "b"), xp, ms, nm, ctypes.byref(prm), st, _stream(stream))
    if check:
        _check(s)
    return [st[i].as_dict() for i in range(nm)]


def profile_enable(g: Gauge, on: bool = True):
    """Reset the live hop-timing counters of g and switch them on or off."""
    _check(_lib.wl_profile_enable(g.handle, int(on)))


def profile_read(g: Gauge) -> dict:
    """Hop launch counters: the inner hop per inner precision ('f64', 'f32',
    'f16') and the outer residual hop ('outer')."""
    arr = (KernelProfile * 4)()
    _check(_lib.wl_profile_read(g.handle, arr))
    return {"f64": arr[0].as_dict(), "f32": arr[1].as_dict(), "f16": arr[2].as_dict(), "outer": arr[3].as_dict()}


def wait_faults(reset: bool = True, stream=None) -> int:
    """Bounded device waits (TMA-staged hops) that gave up since the last reset."""
    n = ctypes.c_uint()
    _check(_lib.wl_wait_faults(ctypes.byref(n), int(reset), _stream(stream)))
    return n.value


VEC_S, VEC_XR, VEC_P, VEC_NORM2 = 0, 1, 2, 3


def vector_op(g: Gauge, kind: int, prec, n_rhs: int, rhs_stride: int, vecs, scal=None, stream=None):
    """wl_vector_op on internal vectors (uint8 CUDA tensors holding n_rhs
    vectors rhs_stride bytes apart); scal: per-rhs (alpha, omega, beta)
    complex triples.  Returns the dots (list) for VEC_XR / VEC_NORM2."""
    vp = (_vp * len(vecs))(*[_ptr(v).value for v in vecs])
    sc = None
    if scal is not None:
        flat = []
        for a, o, b in scal:
            flat += [complex(a).real, complex(a).imag, complex(o).real, complex(o).imag,
                     complex(b).real, complex(b).imag]
        sc = (_dbl * len(flat))(*flat)
    nd = 3 * n_rhs if kind == VEC_XR else n_rhs
    d = (_dbl * nd)()
    _check(_lib.wl_vector_op(g.handle, int(kind), _prec(prec), int(n_rhs), int(rhs_stride), vp, sc, d,
                             _stream(stream)))
    return list(d)


def checked_status(reset: bool = True) -> int:
    """First out-of-range site index recorded by the bounds-checked build
    (0: none; always 0 in the ordinary build)."""
    v = ctypes.c_ulonglong()
    _check(_lib.wl_checked_status(ctypes.byref(v), int(reset)))
    return v.value


def is_checked_build() -> bool:
    return bool(_lib.wl_is_checked_build())


def launch_count() -> int:
    """Kernels launched by the library in this process (wl_launch_count)."""
    n = ctypes.c_longlong()
    _check(_lib.wl_launch_count(ctypes.byref(n)))
    return n.value


HOP_VARIANTS = {"f32": [101, 105, 106, 108, 201, 204, 205, 401, 404, 301, 304, 305, 1104, 1106, 1202, 1203, 5006, 9001,
                        9002, 9004, 9102, 9104],
                "f16": [101, 105, 106, 108, 110, 201, 204, 206, 401, 404, 5006, 9001, 9002, 9004, 9102, 9104],
                "f64": [101, 103, 201, 7101, 7102, 7201, 7202], "df": [101, 103, 104, 105, 106]}


def autotune(g: Gauge, prec, nrhs: int, stream=None):
    """Time every hop variant for (prec, nrhs) and cache the fastest in g.
    Returns (variant, microseconds per launch)."""
    v, us = _int(), _dbl()
    _check(_lib.wl_autotune(g.handle, _prec(prec), int(nrhs), _stream(stream), ctypes.byref(v), ctypes.byref(us)))
    return v.value, us.value


def solve_backward(g: Gauge, b: torch.Tensor, grads, masses, xs=None, prm: SolverParams | None = None,
                   want_links=True, want_masses=True, want_source=True, stream=None):
    """wilson_solve_backward.  Returns (dU (4, V, 8) float64 or None,
    dm0 list or None, db (V, 4, 3) complex128 or None)."""
    prm = prm or params()
    V = g.lat.volume
    nm = len(masses)
    gp = (_vp * nm)(*[_canon(t, V, "g").value for t in grads])
    xp = None
    if xs is not None:
        xp = (_vp * nm)(*[(_canon(x, V, "x").value if x is not None else None) for x in xs])
    ms = (_dbl * nm)(*[float(m) for m in masses])
    dU = torch.zeros((4, V, 8), dtype=torch.float64, device=b.device) if want_links else None
    dm = (_dbl * nm)() if want_masses else None
    db = torch.zeros_like(b) if want_source else None
    _check(_lib.wilson_solve_backward(g.handle, _canon(b, V, "b"), xp, gp, ms, nm, ctypes.byref(prm),
                                      None if dU is None else _ptr(dU), dm,
                                      None if db is None else _ptr(db), _stream(stream)))
    return dU, (list(dm) if dm is not None else None), db


def persistent_selftest(g: Gauge, prec="f32", inject_missing_arrival=False, wait_limit_s=0.05, stream=None) -> int:
    """wl_persistent_selftest: status of one persistent launch (WL_ERR_TIMEOUT when an arrival is withheld)."""
    return _lib.wl_persistent_selftest(g.handle, _prec(prec), int(inject_missing_arrival), float(wait_limit_s),
                                       _stream(stream))
