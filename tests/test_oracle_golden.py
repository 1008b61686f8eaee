"""The oracle reproduces its committed regression fixture and the Table 1 file is well formed."""
import json
import os

import numpy as np

import oracle
from oracle import residuals as R
from paper_2606_29702_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_regression_fixture():
    with open(os.path.join(GOLD, "oracle_burgers_n64.json")) as f:
        ref = json.load(f)
    spec, X, layers = wl.workload("burgers_2x20x4", N=64)
    L, r, grads = oracle.loss_and_grad(R.by_name(spec["family"], **spec["coefs"]), layers, X)
    g = wl.pack(grads)
    np.testing.assert_allclose(L, ref["loss"], rtol=1e-13)
    np.testing.assert_allclose(r[:16, 0], ref["residual_first16"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(g[:32], ref["grad_first32"], rtol=1e-11, atol=1e-15)


def test_table1_fixture():
    with open(os.path.join(GOLD, "table1_ed_vs_ad.json")) as f:
        t = json.load(f)
    assert "Table 1" in t["citation"]
    fp32 = [r for r in t["rows"] if r["dtype"] == "float32"]
    assert len(fp32) == 3 and all(r["residual_rel_l2"] < 1e-6 for r in fp32)
