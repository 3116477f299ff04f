"""Writes tests/golden/tiny_fit.json: the exact optimum of the n=40, p=4
workload (seeded generator, lambda = 2) by brute-force vertex evaluation
(Section 3.2) and the dense simplex (Section 3.1).  Calls only oracle/.
The paper prints no worked example, so these stored values come from the
oracle's exact halves, which the tests also cross-check against each other
and against scipy's LP solver."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2510_15649_gb300 import synth  # noqa: E402


def compute() -> dict:
    """The stored values, computed afresh by the oracle."""
    t = synth.tiny()
    X = t["X"].astype(np.float64)
    y = t["y"].astype(np.float64)
    lam = float(t["lam"])
    fb, bb, nd = oracle.brute_force(X, y, lam)
    fs, bs = oracle.simplex(X, y, lam)
    lmax = oracle.lambda_max(X, y)
    out = dict(workload="n=40 p=4 seed 0 lambda=2", lam=lam, F_star=fb,
               b_star=list(map(float, bb)), n_optimal_vertices=nd,
               F_simplex=fs, lambda_max=lmax,
               source="oracle.brute_force (Section 3.2) / oracle.simplex (Section 3.1)")
    return out


def main():
    out = compute()
    with open(os.path.join(HERE, "tiny_fit.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
