"""The library's monomial tables encode the same PDEs as the oracle's formulas.

Both sides are evaluated on random jets (no network involved): the oracle's
generic monomial evaluator runs the package table, the oracle family runs its
own written-out formula.
"""
import math

import numpy as np
import pytest

from oracle import residuals as R
from paper_2606_29702_gb300 import specs

CASES = [
    ("burgers", dict(nu=0.01 / math.pi)),
    ("ks", dict(c1=1.0, c2=1.0, c4=1.0)),
    ("ks", dict(c1=5.0, c2=0.5, c4=0.005)),
    ("allen_cahn", dict(eps=1e-4, k=5.0)),
    ("helmholtz", dict(k=4 * math.pi)),
    ("ns_psi", dict(nu=0.01)),
    ("ns_uvp", dict(Re=100.0)),
]


@pytest.mark.parametrize("name,coefs", CASES)
def test_spec_matches_oracle_family(name, coefs):
    sp = specs.by_name(name, **coefs)
    fam = R.by_name(name, **coefs)
    fam_m = R.monomial_family(sp.d_in, sp.n_out, sp.components, has_source=sp.has_source)
    g = np.random.default_rng(5)
    N = 40
    X = g.uniform(-1, 1, (N, sp.d_in))
    chans = sorted(set(fam.needed) | set(fam_m.needed))
    jets = {al: g.normal(size=(N, sp.n_out)) for al in chans}
    src = specs.helmholtz_source(X, coefs["k"]) if sp.has_source else None
    a = np.stack(fam.components(jets, X, None if src is None else src[:, 0]), 1)
    b = np.stack(fam_m.components(jets, X, src), 1)
    np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-12)
    assert set(sp.needed()) <= set(fam.needed) | {tuple([0] * sp.d_in)}
