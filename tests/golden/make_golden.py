"""Write oracle_burgers_n64.json from the FP64 oracle (calls only oracle/ and the input generators)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import residuals as R  # noqa: E402
from paper_2606_29702_gb300 import workloads as wl  # noqa: E402


def main():
    spec, X, layers = wl.workload("burgers_2x20x4", N=64)
    fam = R.by_name(spec["family"], **spec["coefs"])
    L, r, grads = oracle.loss_and_grad(fam, layers, X)
    g = wl.pack(grads)
    out = {
        "workload": "burgers_2x20x4 (nu=0.01/pi, 2->20x4->1, Xavier seed 1), first 64 points of seed 0",
        "loss": L,
        "residual_first16": [float(v) for v in r[:16, 0]],
        "grad_first32": [float(v) for v in g[:32]],
        "grad_l2": float((g * g).sum() ** 0.5),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_burgers_n64.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
