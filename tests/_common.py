"""Shared helpers of the test-suite: seeded inputs, oracle references, error metrics."""
import math

import numpy as np

import oracle
from oracle import residuals as R
from paper_2606_29702_gb300 import workloads as wl


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def cosine(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def oracle_family(name, coefs):
    return R.by_name(name, **coefs)


def oracle_source(name, coefs, X):
    """Per-point source the library takes for families with one (Helmholtz f)."""
    if name == "helmholtz":
        return R.helmholtz_source(X, coefs["k"])[:, None]
    return None


def case(name, N, bias_std=0.1, widths=None, seed_shift=0):
    """(spec dict, X, layers, source) for a named workload at N points."""
    spec = dict(wl.WORKLOADS[name])
    if widths is not None:
        spec["widths"] = widths
    X = wl.points(spec["domain"], N, spec["seed_pts"] + seed_shift)
    layers = wl.xavier_layers(spec["widths"], spec["seed_par"] + seed_shift, bias_std)
    return spec, X, layers, oracle_source(spec["family"], spec["coefs"], X)


def reference(spec, X, layers):
    fam = oracle_family(spec["family"], spec["coefs"])
    L, r, g = oracle.loss_and_grad(fam, layers, X)
    return L, r, wl.pack(g)
