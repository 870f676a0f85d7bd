"""Writes the oracle regression fixtures in this folder.

Calls only the FP64 oracle (``oracle/``) on the seeded workloads; the stored
values are a record of the oracle as pinned by the CPU tests, so that a later
change to its arithmetic shows up as a diff here.  Run from the repository
root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2510_07625_gb300 import inputs as I  # noqa: E402


def record(prob, iters, **kw):
    r = O.solve(prob, max_iter=iters, **kw)
    return {
        "seed": prob.seed, "N": prob.N, "dof": prob.model.dof, "iters": iters,
        "X": r["X"].round(12).tolist(), "U": r["U"].round(12).tolist(),
        "alpha_idx": r["alpha_idx"].tolist(), "pcg_iters": r["pcg_iters"].tolist(),
        "kkt_log": [float(f"{v:.12e}") for v in r["kkt_log"]],
        "merit_after": [float(f"{v:.12e}") for v in r["merit_after"]],
    }


def main():
    out = {
        "source": "FP64 oracle, single 7-DoF joint-space solve, seed 0, N=32, dt=0.01, 5 SQP iterations",
        "config_single": record(I.config_single()[0], 5),
        "arm6_seed1_N20": record(I.joint_problem(1, I.arm6(), N=20), 4),
    }
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
