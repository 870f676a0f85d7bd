"""Per-solve rho adaptation (gato_solver_params.rho_adapt; Sec. IV-C adjusts
rho after each SQP iteration from the line search's outcome; here rho / 3
after an accepted step, rho * 2 after a rejected one, within Fig. 4's range
[1e-8, 1e1]) on the GPU.

* fused kernel and plain form agree with the adaptation on (bit for bit for
  the first five iterations of these runs, to FP32 accuracy after);
* an adapted run of K iterations equals K single-iteration calls whose rho is
  set between them by that rule in FP32 (the rule replayed on the host);
* a batch of solves with log-spaced initial rho (the case study's sampling)
  runs in one call, each solve with its own rho.
"""
import dataclasses

import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I
from tests.test_gpu_parity import gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2510_07625_gb300 import gato
    gato.load()
    return gato


def with_rho(p, rho):
    return dataclasses.replace(p, w=tuple(p.w[:5]) + (float(rho),))


def test_rho_adapt_fused_and_plain_agree(G):
    # Both forms follow the rule exactly (next test); they agree bit for bit
    # at rho of order 1e-1 and above, while at rho ~ 4e-4 (the joint cost
    # after five accepted steps from 0.1) one SQP iteration already differs
    # between the two kernels in the last bits (the compiler contracts
    # multiply-adds differently in them), 1e-5 here: held to FP32 accuracy.
    probs = [with_rho(I.ee_problem(1, I.arm7(), 16, 0.05), 1e-3),
             with_rho(I.joint_problem(2, I.arm7(), 12, 0.01), 1e-1)]
    for p in probs:
        a = gpu_solve(G, [p], 6, rho_adapt=1)[0]
        b = gpu_solve(G, [p], 6, plain=True, rho_adapt=1)[0]
        assert a["flags"] == b["flags"]
        for k in ("X", "U"):
            assert np.abs(a[k] - b[k]).max() <= 1e-4 * max(1.0, np.abs(b[k]).max()), k
        a5 = gpu_solve(G, [p], 5, rho_adapt=1)[0]
        b5 = gpu_solve(G, [p], 5, plain=True, rho_adapt=1)[0]
        np.testing.assert_array_equal(a5["X"], b5["X"])


@pytest.mark.parametrize("seed,rho0", [(1, 0.1), (3, 1e-3)])
def test_rho_adapt_replays_the_rule(G, oracle, seed, rho0):
    # FP32 throughout (no precision escalation): a call that escalated would
    # stay in the high-precision mode for its later iterations, which the
    # single-iteration replay, starting every call in FP32, would not
    p = with_rho(I.ee_problem(seed, I.arm7(), 16, 0.05), rho0)
    iters = 8
    full = gpu_solve(G, [p], iters, rho_adapt=1, precision=0)[0]
    X, U, lam = (a.astype(np.float32) for a in oracle.cold_start(p))
    rho = np.float32(rho0)
    outcomes = []
    for _ in range(iters):
        g = gpu_solve(G, [with_rho(p, rho)], 1, X=[X], U=[U], lam=[lam], precision=0)[0]
        accepted = not (g["flags"] & 4)
        outcomes.append(accepted)
        X, U, lam = (g[k].astype(np.float32) for k in ("X", "U", "lam"))
        rho = (np.maximum(rho / np.float32(3.0), np.float32(1e-8)) if accepted
               else np.minimum(rho * np.float32(2.0), np.float32(1e1)))
    assert any(outcomes)
    np.testing.assert_array_equal(full["X"], X)
    np.testing.assert_array_equal(full["U"], U)


def test_log_spaced_rho_batch(G):
    # one start, 16 solves with rho log-spaced over [1e-8, 1e1], adapted; the
    # joint-space cost keeps Q positive definite at any rho (the end-effector
    # cost's Gauss-Newton Q_qq needs rho of order 1 in FP32)
    base = I.joint_problem(5, I.arm7(), 32, 0.05)
    rhos = np.logspace(-8, 1, 16)
    probs = [with_rho(base, r) for r in rhos]
    res = gpu_solve(G, probs, 10, rho_adapt=1)
    for r, g in zip(rhos, res):
        assert np.isfinite(g["X"]).all() and not (g["flags"] & 16), (r, g["flags"])
    # different rho, different paths
    assert len({round(float(g["merit"]), 6) for g in res}) > 1


def test_rho_adapt_with_the_direct_solve(G):
    # the adapted rho reaches the Schur blocks the direct solve eliminates:
    # fused and plain agree bit for bit, and the rule replays like with PCG
    p = with_rho(I.joint_problem(2, I.arm7(), 40, 0.01), 1e-1)
    a = gpu_solve(G, [p], 5, rho_adapt=1, linsolve=1)[0]
    b = gpu_solve(G, [p], 5, plain=True, rho_adapt=1, linsolve=1)[0]
    assert a["flags"] == b["flags"]
    np.testing.assert_array_equal(a["X"], b["X"])
    fixed = gpu_solve(G, [p], 5, rho_adapt=0, linsolve=1)[0]
    assert np.abs(a["X"] - fixed["X"]).max() > 0  # the adaptation changed the path


def test_rho_adapt_against_oracle(G, oracle):
    """An adapted GPU solve against the oracle's adapted solve (Sec. IV-C's
    rule, oracle.solve(rho_adapt=1)).  The first SQP iterations take the
    oracle's line-search decisions (accept/reject drives rho, so the rho
    sequences agree too) unless a decision is a near-tie; run to convergence,
    both reach the same KKT point: X, U within 1e-4, the KKT residuals within
    1e-5 (rho changes the path, not the solution)."""
    from tests.test_gpu_parity import kkt_at, rel

    p = with_rho(I.joint_problem(2, I.arm7(), 32, 0.01), 1e-2)
    g = gpu_solve(G, [p], 6, rho_adapt=1, log=True)[0]
    o = oracle.solve(p, max_iter=6, rho_adapt=1)
    for t in range(6):
        ga, oa = int(g["alpha_idx"][t]), int(o["alpha_idx"][t])
        if ga != oa:
            assert o["merit_gap"][t] <= 1e-5, (t, ga, oa, o["merit_gap"][t])
            break
    gc = gpu_solve(G, [p], 80, rho_adapt=1, kkt_tol=1e-5)[0]
    oc = oracle.solve(p, max_iter=160, rho_adapt=1, kkt_tol=1e-9)
    assert gc["flags"] & 1 and oc["kkt"] <= 1e-7, (gc["flags"], gc["kkt"], oc["kkt"])
    assert rel(gc["X"], oc["X"]) <= 1e-4 and rel(gc["U"], oc["U"]) <= 1e-4
    assert abs(kkt_at(oracle, p, gc["X"], gc["U"], gc["lam"]) - kkt_at(oracle, p, oc["X"], oc["U"], oc["lam"])) <= 1e-5
