"""A constant external end-effector force per solve (gato_problem.f_ext) on
the GPU: Sec. IV-D solves a batch whose problems differ only in the assumed
force and keeps the one whose model best matches the measured motion.

* SQP steps with a force against the oracle's FP64 steps from the same
  iterates (PCG and the direct block elimination);
* fused kernel = plain form, bit for bit, with a force;
* a batch of force hypotheses (directions uniform on the sphere around an
  estimate) in one call: every solve is the one it would be alone, bit for
  bit, and the hypotheses give different solutions.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I
from tests.test_gpu_parity import _per_step_parity, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2510_07625_gb300 import gato
    gato.load()
    return gato


FORCED = [
    ("arm6_fig8_down50", lambda: I.disturbed_ee_problem(0, (0.0, 0.0, -50.0), I.arm6(), 32, 0.01)),
    ("arm7_joint_oblique", lambda: I.disturbed_joint_problem(2, (25.0, -15.0, -40.0), I.arm7(), 24, 0.01)),
]


@pytest.mark.parametrize("name,mk", FORCED, ids=[f[0] for f in FORCED])
def test_forced_per_step_parity(G, oracle, name, mk):
    _per_step_parity(G, oracle, mk(), 4)


def test_forced_per_step_parity_direct(G, oracle):
    _per_step_parity(G, oracle, FORCED[0][1](), 3, linsolve=1)


def test_forced_fused_equals_plain_bitwise(G):
    for _, mk in FORCED:
        p = mk()
        a = gpu_solve(G, [p], 3)[0]
        b = gpu_solve(G, [p], 3, plain=True)[0]
        assert a["flags"] == b["flags"]
        for k in ("X", "U", "lam"):
            np.testing.assert_array_equal(a[k], b[k])


def test_force_hypothesis_batch(G, oracle):
    M = 16
    F = I.force_hypotheses(7, M, center=(0.0, 0.0, -30.0), radius=20.0)
    probs = [I.disturbed_ee_problem(0, f, I.arm6(), 32, 0.01) for f in F]
    batch = gpu_solve(G, probs, 3)
    for j in (0, 5, 15):
        alone = gpu_solve(G, [probs[j]], 3)[0]
        assert alone["flags"] == batch[j]["flags"]
        for k in ("X", "U", "lam"):
            np.testing.assert_array_equal(alone[k], batch[j][k])
    U0 = np.stack([g["U"] for g in batch])
    spread = np.abs(U0 - U0[0]).max(axis=(1, 2))
    assert (spread[1:] > 1e-2).all()  # every hypothesis moves the controls
    # one step of two hypotheses against the oracle: the same step length
    # (unless a near-tie) and the step within its FP32 accuracy
    from tests.test_gpu_parity import STEP_TOL, _step_error
    for j in (0, 9):
        g = gpu_solve(G, [probs[j]], 1, log=True)[0]
        X, U, lam = oracle.cold_start(probs[j])
        o = oracle.solve(probs[j], max_iter=1, X=X, U=U, lam=lam)
        ga, oa = int(g["alpha_idx"][0]), int(o["alpha_idx"][0])
        if o["merit_gap"][0] > 1e-5:
            assert ga == oa, (j, ga, oa)
        if ga == oa and oa >= 0:
            assert _step_error(X, U, g, o) <= STEP_TOL, j


def test_forced_direct_fused_equals_plain_bitwise(G):
    p = FORCED[0][1]()
    a = gpu_solve(G, [p], 3, linsolve=1)[0]
    b = gpu_solve(G, [p], 3, plain=True, linsolve=1)[0]
    assert a["flags"] == b["flags"]
    for k in ("X", "U", "lam"):
        np.testing.assert_array_equal(a[k], b[k])
