"""Shared test helpers: seeded inputs, canonical/torch conversion, error norms."""
import numpy as np


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


TOL = {"f64": 1e-12, "df": 1e-12, "f32": 1e-6, "f16": 5e-3}


def neighbour_sites(dims, sites):
    """Sorted lexicographic sites n and n +- mu (periodic wrap) for n in sites."""
    X, Y, Z, T = dims
    ext = np.array(dims)
    sites = np.asarray(sites, dtype=np.int64)
    c = np.stack([sites % X, (sites // X) % Y, (sites // (X * Y)) % Z, sites // (X * Y * Z)], axis=1)
    out = [sites]
    for mu in range(4):
        for d in (1, -1):
            cm = c.copy()
            cm[:, mu] = (cm[:, mu] + d) % ext[mu]
            out.append(cm[:, 0] + X * (cm[:, 1] + Y * (cm[:, 2] + Z * cm[:, 3])))
    return np.unique(np.concatenate(out))


class SampledResidual:
    """FP64 oracle residual r = b - M_k(m) x of a solution at sampled sites,
    for lattices too large for an oracle solve or a full oracle matvec.

    Two figures per solution, both relative to ||b||:
      est  -- ||r|| over n_random uniformly drawn sites, scaled by
              sqrt(V / n_random): an unbiased estimate of the true residual;
      peak -- the largest single-site ||r_n|| over those sites and the
              point-source site with its eight neighbours; never above the
              true relative residual.
    x may be a CUDA tensor: only the sites the stencil reads are copied."""

    def __init__(self, dims, U, n_random=4096, seed=0, source_site=0):
        V = int(np.prod(dims))
        rng = np.random.default_rng(seed)
        self.random = np.unique(rng.choice(V, size=min(n_random, V), replace=False))
        self.sites = np.unique(np.concatenate([self.random, neighbour_sites(dims, [source_site])]))
        self.is_random = np.isin(self.sites, self.random)
        self.need = neighbour_sites(dims, self.sites)
        self.dims, self.U, self.V = dims, U, V
        self.psi = np.zeros((V, 4, 3), dtype=np.complex128)

    def __call__(self, x, b, m):
        import torch
        from oracle import oracle as O
        idx = torch.from_numpy(self.need)
        if isinstance(x, torch.Tensor):
            self.psi[self.need] = x[idx.to(x.device)].cpu().numpy()
        else:
            self.psi[self.need] = x[self.need]
        r = b[self.sites] - O.apply_mk_sites(self.U, self.dims, self.psi, O.kappa(m), self.sites)
        bn = float(np.linalg.norm(b))
        rr = r[self.is_random].reshape(-1)
        est = float(np.linalg.norm(rr)) * np.sqrt(self.V / int(self.is_random.sum())) / bn
        peak = float(np.max(np.linalg.norm(r.reshape(len(self.sites), -1), axis=1))) / bn
        return est, peak
