"""Write tests/golden/oracle_counts.json from the CPU oracle only.

Run:  python tests/golden/make_golden.py
The stored values are per-level PCG iteration and call counts and the norm of
the solution for small versions of the three single-problem workloads.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_math_9809043_gb300 import problems as P  # noqa: E402

CASES = [
    {"config": 0, "scale": None, "tol": 1e-8},
    {"config": 1, "scale": 128, "tol": 1e-8},
    {"config": 2, "scale": 16, "tol": 1e-8},
]


def main():
    out = {"generator": "tests/golden/make_golden.py (CPU oracle)", "cases": []}
    for c in CASES:
        prob = P.config_problem(c["config"], scale=c["scale"])
        H = O.Hierarchy(prob)
        x, st = H.solve(H.lift_rhs(), c["tol"])
        assert st["status"] == 0, st
        out["cases"].append({**c, "dims": H.dims, "iters": st["iters"], "calls": st["calls"],
                             "xnorm": float(np.linalg.norm(x)), "relres_true": st["relres_true"]})
        print(c, st["iters"], st["calls"])
    with open(os.path.join(HERE, "oracle_counts.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
