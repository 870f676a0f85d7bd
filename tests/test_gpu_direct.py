"""The direct linear solve (gato_solver_params.linsolve = GATO_LINSOLVE_DIRECT):
S dnu = rhs by block elimination from both ends of the horizon instead of
PCG (GPU).

* on the GPU's own Schur system, read back and solved densely in FP64: the
  block elimination is backward stable for SPD S, so its error is bounded by
  the condition of S times FP32 rounding; the bar is the PCG stage test's
  5e-3 and the measured error is far below it;
* the fused kernel equals the plain form bit for bit, and one SQP step is
  the same bit for bit for every split of the knots over a cluster (the two
  ends meet at m = floor((N+1)/2) whatever the split, so every knot's
  operations are the same; the step's merit sums differ only in order, which
  picks the same alpha).  N = 63 puts m on a CTA's first knot for 8 and 4
  CTAs, N = 64 on the first CTA's last knot for 2;
* each SQP step against the oracle's step with its direct solver (the
  per-step bound of the PCG parity tests).
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I
from tests.test_gpu_parity import _per_step_parity, gpu_solve
from tests.test_gpu_stages import PROBS, V_DNU, V_RHS, block, midpoint, stage, vec

pytestmark = pytest.mark.gpu

DIRECT = 1


@pytest.fixture(scope="module")
def G():
    from paper_2510_07625_gb300 import gato
    gato.load()
    return gato


@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_direct_solve_stage(G, oracle, name, mk):
    from tests.test_oracle_kkt import blocks_to_dense
    prob = mk()
    X, U, lam = midpoint(oracle, prob)
    N, K = prob.N, prob.N + 1
    buf, off, _ = stage(G, prob, 9, X, U, lam, linsolve=DIRECT)
    D = block(buf, off, "D", K)
    L = block(buf, off, "L", K)
    rhs = vec(buf, off, N, V_RHS).ravel()
    dnu = vec(buf, off, N, V_DNU).ravel()
    Sg = blocks_to_dense(D, L[1:])
    exact = np.linalg.solve(Sg, rhs)
    err = np.abs(dnu - exact).max() / np.abs(exact).max()
    assert err < 5e-3, err
    # the residual of the FP32 solution on the FP32 system, relative to |S||x|
    res = np.abs(Sg @ dnu - rhs).max() / (np.abs(Sg).max() * np.abs(dnu).max())
    assert res < 1e-5, res


def test_direct_fused_equals_plain_bitwise(G):
    probs = [I.joint_problem(0, I.arm7(), N=16), I.ee_problem(1, I.arm7(), N=12),
             I.joint_problem(2, I.arm6(), N=9)]
    for p in probs:
        a = gpu_solve(G, [p], 3, linsolve=DIRECT)[0]
        b = gpu_solve(G, [p], 3, plain=True, linsolve=DIRECT)[0]
        for k in ("X", "U", "lam"):
            np.testing.assert_array_equal(a[k], b[k])
        assert a["pcg_iters"] == 0 and b["pcg_iters"] == 0


@pytest.mark.parametrize("launch", [(1, 9, 0), (1, 0, 4), (2, 0, 0), (1, 17, 0)],
                         ids=["kpc9", "uniform4", "throughput", "kpc17"])
def test_direct_step_independent_of_the_split(G, launch):
    probs = [I.ee_problem(4, I.arm7(), 64), I.joint_problem(5, I.arm7(), 64, 0.01),
             I.joint_problem(6, I.arm7(), 63, 0.01)]
    a = gpu_solve(G, probs, 1, launch=(1, 0, 0), linsolve=DIRECT)
    b = gpu_solve(G, probs, 1, launch=launch, linsolve=DIRECT)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x["X"], y["X"])
        np.testing.assert_array_equal(x["U"], y["U"])
        np.testing.assert_array_equal(x["lam"], y["lam"])


def test_direct_per_step_parity(G, oracle):
    for p in (I.joint_problem(0, I.arm7(), 32, 0.01), I.ee_problem(3, I.arm7(), 24, 0.01)):
        _per_step_parity(G, oracle, p, 4, linsolve=DIRECT)
