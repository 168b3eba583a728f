"""Seeded synthetic inputs: gauge fields and sources.

This module is the only code shared by the CUDA path's tests/benchmarks and
the FP64 oracle.  It holds input generation only -- none of the Wilson
operator's or the solvers' arithmetic.

Random numbers come from a counter-based generator: the splitmix64 finaliser
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to (seed, stream, counter).  Every value is a pure
function of its key, so any subset of a field can be regenerated without
drawing the rest.

Canonical layouts (complex128, lexicographic site n = x + X*(y + Y*(z + Z*t))):
  spinor  [site][spin 4][colour 3]
  links   [mu 4][site][row 3][col 3], mu = 0..3 <-> x, y, z, t

Gauge links follow the recipe U = exp(i*eps*H), H = sum_a c_a lambda_a / 2
with c_a ~ N(0, 1) and lambda_a the Gell-Mann matrices, computed through the
Hermitian eigendecomposition of H in FP64, then re-orthonormalised so that
row 2 = conj(row 0 x row 1) holds to rounding (U in SU(3)).
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import shared_memory

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

# stream ids, one per kind of draw
STREAM_GAUGE = 0
STREAM_Z2 = 1
STREAM_GAUSS = 2
STREAM_GAUGE_TRANSFORM = 3
STREAM_DIRECTION = 4


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function (wrapping uint64 arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """64 random bits for each counter value under key (seed, stream)."""
    counter = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.uint64(stream + 1))
        return _mix(key + _GOLDEN * (counter + np.uint64(1)))


def uniform(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1]: top 53 bits, shifted away from zero."""
    bits = u64(seed, stream, counter) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Standard normals by Box-Muller (cosine branch) from counters 2k, 2k+1."""
    counter = np.asarray(counter, dtype=np.uint64)
    u1 = uniform(seed, stream, counter * np.uint64(2))
    u2 = uniform(seed, stream, counter * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
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


def volume(dims) -> int:
    X, Y, Z, T = dims
    return int(X) * int(Y) * int(Z) * int(T)


def _reunitarize(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt rows 0 and 1, then row 2 = conj(row0 x row1)."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def su3_from_coeffs(c: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*sum_a c_a lambda_a/2) for coefficient arrays of shape (..., 8)."""
    H = np.einsum("...a,aij->...ij", c, gell_mann() / 2.0)
    w, V = np.linalg.eigh(H)
    U = np.einsum("...ik,...k,...jk->...ij", V, np.exp(1j * eps * w), np.conj(V))
    return _reunitarize(U)


def _gauge_chunk(flat: np.ndarray, start: int, stop: int, eps: float, seed: int) -> None:
    link = np.arange(start, stop, dtype=np.uint64)  # link = mu*V + site
    ctr = link[:, None] * np.uint64(8) + np.arange(8, dtype=np.uint64)[None, :]
    flat[start:stop] = su3_from_coeffs(normal(seed, STREAM_GAUGE, ctr), eps)


def _gauge_worker(args) -> None:
    name, n_links, starts, chunk, eps, seed = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        flat = np.ndarray((n_links, 3, 3), dtype=np.complex128, buffer=shm.buf)
        for start in starts:
            _gauge_chunk(flat, start, min(n_links, start + chunk), eps, seed)
        del flat
    finally:
        shm.close()


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 20, workers: int | None = None) -> np.ndarray:
    """Random SU(3) links U_mu(n) = exp(i eps H), canonical layout (4, V, 3, 3).

    Every link is a pure function of (seed, link index), so the field is the
    same for any chunking.  Fields of 8M links or more are generated by
    ``workers`` spawned processes (default: one per core, at most 16) writing
    into shared memory."""
    V = volume(dims)
    n_links = 4 * V
    starts = list(range(0, n_links, chunk))
    if workers is None:
        workers = min(16, os.cpu_count() or 1, len(starts)) if n_links >= (1 << 23) else 1
    if workers <= 1:
        out = np.empty((4, V, 3, 3), dtype=np.complex128)
        flat = out.reshape(n_links, 3, 3)
        for start in starts:
            _gauge_chunk(flat, start, min(n_links, start + chunk), eps, seed)
        return out
    shm = shared_memory.SharedMemory(create=True, size=n_links * 9 * 16)
    try:
        jobs = [(shm.name, n_links, starts[w::workers], chunk, eps, seed) for w in range(workers)]
        # a worker that dies raises BrokenProcessPool here instead of being respawned
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_gauge_worker, jobs))
        out = np.ndarray((4, V, 3, 3), dtype=np.complex128, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return out


def unit_gauge_field(dims) -> np.ndarray:
    """Free field U = 1."""
    V = volume(dims)
    out = np.zeros((4, V, 3, 3), dtype=np.complex128)
    out[..., 0, 0] = out[..., 1, 1] = out[..., 2, 2] = 1.0
    return out


def random_gauge_transform(dims, seed: int, eps: float = 3.0) -> np.ndarray:
    """Random SU(3) matrix g(n) per site, shape (V, 3, 3)."""
    V = volume(dims)
    ctr = np.arange(V, dtype=np.uint64)[:, None] * np.uint64(8) + np.arange(8, dtype=np.uint64)[None, :]
    return su3_from_coeffs(normal(seed, STREAM_GAUGE_TRANSFORM, ctr), eps)


def point_source(dims, spin: int = 0, colour: int = 0, site: int = 0) -> np.ndarray:
    """Unit point source, canonical spinor layout (V, 4, 3)."""
    b = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def z2_source(dims, seed: int) -> np.ndarray:
    """Z2 noise: independent +-1 on the real and imaginary part of every entry."""
    n = volume(dims) * 12
    bits = u64(seed, STREAM_Z2, np.arange(2 * n, dtype=np.uint64)) >> np.uint64(63)
    pm = 1.0 - 2.0 * bits.astype(np.float64)
    return (pm[0::2] + 1j * pm[1::2]).reshape(volume(dims), 4, 3)


def gaussian_source(dims, seed: int) -> np.ndarray:
    """Complex Gaussian source: real and imaginary parts independent N(0, 1)."""
    n = volume(dims) * 12
    g = normal(seed, STREAM_GAUSS, np.arange(2 * n, dtype=np.uint64))
    return (g[0::2] + 1j * g[1::2]).reshape(volume(dims), 4, 3)


def su3_directions(dims, seed: int) -> np.ndarray:
    """Random su(3) coefficient fields, shape (4, V, 8), entries N(0, 1)."""
    V = volume(dims)
    ctr = np.arange(4 * V * 8, dtype=np.uint64)
    return normal(seed, STREAM_DIRECTION, ctr).reshape(4, V, 8)


def lex_coords(dims) -> np.ndarray:
    """(V, 4) integer coordinates (x, y, z, t) of each lexicographic site."""
    X, Y, Z, T = dims
    n = np.arange(volume(dims))
    return np.stack([n % X, (n // X) % Y, (n // (X * Y)) % Z, n // (X * Y * Z)], axis=1)


def parity(dims) -> np.ndarray:
    """Site parity (x+y+z+t) mod 2 of each lexicographic site."""
    return lex_coords(dims).sum(axis=1) % 2
