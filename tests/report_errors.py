"""Error of the FP32 GPU solver against the FP64 oracle, per workload (GPU).

Run as ``python tests/report_errors.py`` on a machine with the GPU; prints one
JSON object per workload with, for each solve, the relative X and U errors
after the workload's fixed iteration count (same cold start on both sides)
and after convergence (both solved to their floors), plus the KKT residuals.
Relative error = max |GPU - oracle| / max(1, max |oracle|).  The end-effector
cost has no term in the joint positions beyond the end-effector position
(a 7-DoF arm tracking a 3-D point), so its minimisers are not unique in X;
for those workloads the merit of both iterates (evaluated by the oracle)
and the KKT residuals are the comparable quantities.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2510_07625_gb300 import gato as G, inputs as I  # noqa: E402
from tests.test_gpu_parity import gpu_solve, rel  # noqa: E402


def errors(probs, iters, converge_iters, **prm):
    out = []
    g_fix = gpu_solve(G, probs, iters, **prm)
    g_conv = gpu_solve(G, probs, converge_iters, **prm)
    for p, gf, gc in zip(probs, g_fix, g_conv):
        of = O.solve(p, max_iter=iters)
        oc = O.solve(p, max_iter=converge_iters + 60, kkt_tol=1e-9)
        # the merit of each side's iterate, both evaluated by the oracle in FP64
        mf = (O.merit(p, gf["X"], gf["U"]), O.merit(p, of["X"], of["U"]))
        mc = (O.merit(p, gc["X"], gc["U"]), O.merit(p, oc["X"], oc["U"]))
        out.append({"seed": p.seed, "N": p.N, "dof": p.model.dof,
                    "fixed": {"iters": iters, "eX": rel(gf["X"], of["X"]), "eU": rel(gf["U"], of["U"]),
                              "merit_rel": abs(mf[0] - mf[1]) / abs(mf[1]),
                              "kkt_gpu": gf["kkt"], "kkt_oracle": of["kkt"]},
                    "converged": {"eX": rel(gc["X"], oc["X"]), "eU": rel(gc["U"], oc["U"]),
                                  "merit_rel": abs(mc[0] - mc[1]) / abs(mc[1]),
                                  "kkt_gpu": gc["kkt"], "kkt_oracle": oc["kkt"], "flags": gc["flags"]}})
    return out


def summary(name, rows):
    f = [max(r["fixed"]["eX"], r["fixed"]["eU"]) for r in rows]
    c = [max(r["converged"]["eX"], r["converged"]["eU"]) for r in rows]
    k = [r["converged"]["kkt_gpu"] for r in rows]
    mf = [r["fixed"]["merit_rel"] for r in rows]
    mc = [r["converged"]["merit_rel"] for r in rows]
    ko = [r["converged"]["kkt_oracle"] for r in rows]
    return {"workload": name, "solves": len(rows),
            "fixed_count_err_median": float(np.median(f)), "fixed_count_err_max": float(np.max(f)),
            "fixed_count_merit_rel_max": float(np.max(mf)),
            "converged_err_median": float(np.median(c)), "converged_err_max": float(np.max(c)),
            "converged_merit_rel_max": float(np.max(mc)),
            "converged_kkt_gpu_max": float(np.max(k)), "converged_kkt_oracle_max": float(np.max(ko))}


def main():
    O.build()
    G.load()
    runs = [
        ("single solve: 7-DoF joint cost, N=32, 5 iterations", [I.joint_problem(0, I.arm7(), 32, 0.01)], 5, 40),
        ("fixed batch: 7-DoF joint cost, N=32, seeds 0..7 of 32, 10 iterations",
         [I.joint_problem(s, I.arm7(), 32, 0.01) for s in range(8)], 10, 40),
        ("sweep: figure-eight EE, seeds 0..3, N=32/64/128, 10 iterations",
         [I.ee_problem(s, I.arm7(), N) for N in (32, 64, 128) for s in range(4)], 10, 60),
        ("uneven mix: first 8 of 128 (N 16..128, 7/6-DoF), 20 iterations", I.config_uneven(B=8), 20, 80),
    ]
    for name, probs, it, conv in runs:
        rows = errors(probs, it, conv)
        print(json.dumps(summary(name, rows)), flush=True)


if __name__ == "__main__":
    main()
