"""Shared test helpers: seeded inputs, canonical/torch conversion, error norms."""
import numpy as np


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


TOL = {"f64": 1e-12, "df": 1e-12, "f32": 1e-6, "f16": 5e-3}
