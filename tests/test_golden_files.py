"""The stored oracle results under tests/golden, written by
make_oracle_multimass.py from oracle/ alone: their workload metadata match
the script's workloads, every record covers every mass at the 1e-10
tolerance with its polished solution at every stored site, and the
solution at the point source's own site and component is what the
hopping expansion of x = (1 - kappa D)^-1 b gives there for the heaviest
mass: 1 plus closed paths back to the site, of which those of two hops
vanish ((1 - gamma_mu)(1 + gamma_mu) = 0, Eq. 4), so 1 + O(kappa^4) -- the
kappa normalisation of Eq. 3 (the paper's psi = x / (m0 + 4) would be near
0.22), at the right site and component."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _script():
    spec = importlib.util.spec_from_file_location("make_oracle_multimass",
                                                  os.path.join(GOLDEN, "make_oracle_multimass.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("config", ["c3", "c5"])
def test_stored_oracle_runs_are_complete_and_consistent(config):
    path = os.path.join(GOLDEN, f"{config}_oracle_multimass.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle run for {config}")
    gold = json.load(open(path))
    w = _script().WORKLOADS[config]
    assert tuple(gold["dims"]) == tuple(w["dims"]) and gold["eps"] == w["eps"] and gold["gauge_seed"] == w["seed"]
    assert gold["masses"] == w["masses"] and gold["tol"] == 1e-10 and gold["polish_tol"] == 1e-13
    X, Y, Z, T = gold["dims"]
    sites = gold["sites"]
    assert sites == sorted(set(sites)) and sites[0] == 0 and all(0 <= s < X * Y * Z * T for s in sites)
    # the source site and its eight neighbours are always kept
    for mu, ext in enumerate(gold["dims"]):
        for d in (1, ext - 1):
            c = [0, 0, 0, 0]
            c[mu] = d
            assert c[0] + X * (c[1] + Y * (c[2] + Z * c[3])) in sites
    n_mass = len(gold["masses"])
    assert gold["sources"]
    for key, rec in gold["sources"].items():
        k = int(key)
        assert 0 <= k < 12
        assert len(rec["iterations"]) == n_mass and all(isinstance(v, int) and v > 0 for v in rec["iterations"])
        assert all(0 < r <= 1e-10 for r in rec["true_relres"])
        assert len(rec["x"]) == n_mass
        for x in rec["x"]:
            a = np.array(x)
            assert a.shape == (len(sites), 12, 2) and np.all(np.isfinite(a))
        # heaviest mass: x at the source site and component = 1 + O(kappa^4)
        # (48 closed four-hop paths through a site, plus longer ones)
        kappa = 1.0 / (2.0 * gold["masses"][0] + 8.0)
        z = complex(*rec["x"][0][0][k])
        assert abs(z - 1.0) < 256 * kappa ** 4, (key, z)
