"""The closed-loop hypothesize-and-test harness (Sec. IV-D) on the CPU: the
plant is the library's host RK4 plant, the batch solver the FP64 oracle (a
test stand-in for the GPU solve), the latency fixed.

* the selection keeps exactly the true force when it is among the candidates
  (the hypothesis' model is then the plant itself);
* with the true force as the initial estimate every tick keeps hypothesis 0
  and the estimate stays exact;
* with an unknown force the estimate moves toward it.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import closed_loop as CL
from paper_2510_07625_gb300 import inputs as I


@pytest.fixture(scope="module")
def plant():
    from paper_2510_07625_gb300 import build, gato

    build.build_library()
    gato.load()
    return gato.Plant(I.arm6())


def oracle_solver(oracle, default_iters=2):
    def solve(probs, X, U, lam, iters=None):
        it = iters or default_iters
        out = []
        for i, p in enumerate(probs):
            n = p.model.dof
            r = oracle.solve(p, max_iter=it,
                             X=None if X is None else np.asarray(X[i], np.float64),
                             U=None if U is None else np.asarray(U[i], np.float64),
                             lam=None if lam is None else np.asarray(lam[i], np.float64))
            out.append(dict(X=r["X"].reshape(p.N + 1, 2 * n), U=r["U"].reshape(p.N, n),
                            lam=r["lam"].reshape(p.N + 1, 2 * n), flags=r["flags"]))
        return out, 0.0
    return solve


def test_selection_recovers_the_true_force(plant):
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 6)])
    u = rng.uniform(-20, 20, 6)
    F = I.force_hypotheses(11, 8, center=(0.0, 0.0, -30.0), radius=15.0)
    for j in (0, 3, 7):
        meas = plant.rk4(x, u, 1e-3, 4, f_ext=F[j])
        assert CL.select_hypothesis(plant, x, u, 4, 1e-3, F, meas) == j


def test_known_force_is_kept(plant, oracle):
    f = (0.0, 0.0, -40.0)
    r = CL.run(oracle_solver(oracle), plant, 4, f, N=8, sim_s=0.02, latency_s=0.004, settle_s=0.0,
               warm_iters=5, f0=f)
    assert r.ticks == 5 and r.picks == [0] * 5
    assert r.f_err == 0.0
    assert np.isfinite(r.track_err_mean)


def test_estimate_moves_toward_an_unknown_force(plant, oracle):
    f = np.array([0.0, 0.0, -50.0])
    r = CL.run(oracle_solver(oracle), plant, 8, f, N=8, sim_s=0.04, latency_s=0.004, settle_s=0.0,
               radius=15.0, warm_iters=5)
    assert r.f_err < 0.8 * np.linalg.norm(f)


def test_selection_skips_failed_solves(plant):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 6)])
    u = rng.uniform(-20, 20, 6)
    F = I.force_hypotheses(12, 6, center=(0.0, 0.0, -30.0), radius=15.0)
    meas = plant.rk4(x, u, 1e-3, 3, f_ext=F[2])
    assert CL.select_hypothesis(plant, x, u, 3, 1e-3, F, meas, usable={0, 1, 3, 4, 5}) != 2
    assert CL.select_hypothesis(plant, x, u, 3, 1e-3, F, meas, usable=set()) is None
