"""Mass sets placed relative to the critical mass, and the single-mass versus
multi-shift comparison of the paper's Section 7 on synthetic fields.

The paper measures on a quenched ensemble whose critical mass is
am_c = -0.8173 and uses two mass sets (Table 2): a wide one and a narrow one
close to m_c. Our synthetic fields have their own m_c, so the sets are
placed at the paper's distances m - m_c from it:

- `critical_mass` finds the rightmost eigenvalue mu_max of the hop D by
  Krylov-Schur restarted Arnoldi, with the library's FP64 dslash as the
  operator and the basis on the GPU. M_p(m) = (m + 4) - D/2 has eigenvalues (m + 4) - mu/2, so
  its real parts reach zero first at m_c = Re(mu_max)/2 - 4, and the
  conditioning of a solve at m grows like 1/(m - m_c). For U = 1 with an
  antiperiodic time direction, m_c = cos(pi/T) - 1.
- `table2_sets` shifts the paper's two sets to a given m_c.
- `main` solves both sets with the single-mass scheme (zero guess and
  Lagrange guess) and with BiCGstab-M (vectors and hops in double-float
  and in FP64), and prints one JSON line per set with each solver's
  iterations, seconds and speed-up over the faster BiCGstab-M (the
  quantities of Table 3).

python -m paper_1103_5103_gb300.mass_sets [--dims 16x16x16x32] [--eps 0.5] [--sources z2|point]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import api, synth

PAPER_MC = -0.8173
PAPER_WIDE = [-0.7908, -0.7721, -0.7511, -0.7320, -0.7105, -0.6193, -0.5108, -0.2687]
PAPER_NARROW = [-0.7908, -0.7887, -0.7866, -0.7846, -0.7825, -0.7804, -0.7784, -0.7763]


def rightmost_eigenvalue(matvec, v0: torch.Tensor, tol: float = 1e-6, m: int = 64, k: int = 24,
                         max_restarts: int = 400):
    """The eigenvalue with the largest real part of a complex linear operator,
    by Krylov-Schur restarted Arnoldi (Stewart, SIAM J. Matrix Anal. Appl. 23,
    2001): expand an orthonormal basis to m vectors (classical Gram-Schmidt,
    applied twice), take the complex Schur form of the projected matrix,
    keep the k Schur vectors whose Ritz values lie furthest right, and
    continue from them.  matvec maps a 1-D complex128 tensor to one of the
    same shape (on v0's device).  Returns (eigenvalue, converged, products):
    converged when the residual of the rightmost Ritz pair is below
    tol * |eigenvalue|; otherwise the best Ritz value after max_restarts."""
    from scipy.linalg import schur
    n = v0.numel()
    m = min(m, n - 1)
    k = min(k, m - 2)
    V = torch.zeros((m + 1, n), dtype=torch.complex128, device=v0.device)
    V[0] = v0.reshape(-1) / torch.linalg.vector_norm(v0)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    p, products, best = 0, 0, None
    for _ in range(max_restarts):
        for j in range(p, m):
            w = matvec(V[j])
            products += 1
            h = V[:j + 1].conj() @ w
            w = w - h @ V[:j + 1]
            h2 = V[:j + 1].conj() @ w
            w = w - h2 @ V[:j + 1]
            beta = float(torch.linalg.vector_norm(w))
            H[:j + 1, j] = (h + h2).cpu().numpy()
            H[j + 1, j] = beta
            V[j + 1] = w / beta
        ev = np.linalg.eigvals(H[:m, :m])
        thr = np.sort(ev.real)[::-1][k - 1]
        T, Z, kk = schur(H[:m, :m], output="complex", sort=lambda x: x.real >= thr)
        b = H[m, m - 1] * Z[m - 1, :kk]
        theta, Y = np.linalg.eig(T[:kk, :kk])
        i = int(np.argmax(theta.real))
        best = complex(theta[i])
        if abs(b @ Y[:, i]) / np.linalg.norm(Y[:, i]) <= tol * abs(best):
            return best, True, products
        # truncate to the kk wanted Schur vectors: A V_k = V_k T_k + v_{k+1} b^T
        V[:kk] = torch.from_numpy(np.ascontiguousarray(Z[:, :kk].T)).to(V.device) @ V[:m]
        V[kk] = V[m]
        H[:] = 0
        H[:kk, :kk] = T[:kk, :kk]
        H[kk, :kk] = b
        p = kk
    return best, False, products


def critical_mass(g: api.Gauge, seed: int = 11, tol: float = 1e-6, max_restarts: int = 400):
    """(m_c, converged, products): m_c = Re(mu_max)/2 - 4, mu_max the
    rightmost eigenvalue of D, with the library's FP64 dslash as the
    operator and the Krylov basis kept on the GPU."""
    dims = g.lat.dims
    V = g.lat.volume
    out = torch.empty((V, 4, 3), dtype=torch.complex128, device="cuda")

    def hop(x):
        api.wilson_dslash(g, x.reshape(V, 4, 3), out, 0.0, "f64", api.OP_HOP)
        return out.reshape(-1).clone()

    v0 = torch.from_numpy(synth.gaussian_source(dims, seed=seed)).cuda().reshape(-1)
    mu, ok, nprod = rightmost_eigenvalue(hop, v0, tol, max_restarts=max_restarts)
    return mu.real / 2.0 - 4.0, ok, nprod


def table2_sets(m_c: float):
    """The paper's wide and narrow sets at the same distances from m_c."""
    wide = [m_c + (m - PAPER_MC) for m in PAPER_WIDE]
    narrow = [m_c + (m - PAPER_MC) for m in PAPER_NARROW]
    return wide, narrow


def run(dims, eps, seed, kind, inner, repeat=2):
    lat = api.Lattice(dims)
    U = torch.from_numpy(synth.gauge_field(dims, eps, seed=seed)).cuda()
    g = api.Gauge(lat, U)
    t0 = time.perf_counter()
    m_c, mc_converged, mc_products = critical_mass(g, tol=1e-6)
    t_mc = time.perf_counter() - t0
    b = synth.point_source(dims) if kind == "point" else synth.z2_source(dims, seed=seed + 1)
    bd = torch.from_numpy(b).cuda()
    shadow = torch.from_numpy(synth.gaussian_source(dims, seed=seed + 2)).cuda() if kind == "point" else None
    wide, narrow = table2_sets(m_c)
    rows = []
    for name, masses in (("wide", wide), ("narrow", narrow)):
        res = {}
        for label, prm in (("single-mass, zero guess", api.params(guess=api.GUESS_ZERO, inner_prec=inner)),
                           ("single-mass, Lagrange guess", api.params(guess=api.GUESS_POLY, inner_prec=inner))):
            for _ in range(repeat):
                torch.cuda.synchronize()
                t = time.perf_counter()
                _, st = api.multimass_solve(g, [bd], masses, prm)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
            res[label] = {"iterations": sum(s["iterations"] for s in st[0]), "seconds": dt,
                          "ms_per_iteration": 1e3 * dt / max(1, sum(s["iterations"] for s in st[0])),
                          "max_true_relres": max(s["true_relres"] for s in st[0])}
        xs = [torch.empty_like(bd) for _ in masses]
        t_ms = []
        for label, outer in (("multi-shift (BiCGstab-M, double-float)", "df"),
                             ("multi-shift (BiCGstab-M, FP64)", "f64")):
            for _ in range(repeat):
                torch.cuda.synchronize()
                t = time.perf_counter()
                stm = api.bicgstab_m_solve(g, bd, xs, masses, api.params(shadow=shadow, outer_prec=outer),
                                           check=False)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
            it_m = max(s["iterations"] for s in stm)
            res[label] = {"iterations": it_m, "seconds": dt, "ms_per_iteration": 1e3 * dt / max(1, it_m),
                          "max_true_relres": max(s["true_relres"] for s in stm),
                          "masses_polished": sum(1 for s in stm if s["restarts"] > 0)}
            t_ms.append(dt)
        for label, r in res.items():
            r["speed_up_vs_multi_shift"] = min(t_ms) / r["seconds"]
        row = {"dims": "x".join(map(str, dims)), "eps": eps, "source": kind, "inner": inner, "m_c": m_c,
               "m_c_converged": mc_converged, "m_c_products": mc_products, "m_c_seconds": t_mc, "set": name, "masses": masses, "results": res}
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="16x16x16x32")
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--sources", choices=["z2", "point"], default="z2")
    ap.add_argument("--inner", choices=["f32", "f16", "f64"], default="f32")
    args = ap.parse_args()
    run(tuple(int(v) for v in args.dims.split("x")), args.eps, args.seed, args.sources, args.inner)


if __name__ == "__main__":
    main()
