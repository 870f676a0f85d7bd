"""Pins for the oracle's SQP loop (Sec. II-A Steps 1-3, Eq. 3 and Eq. 7).

* LQR special case: a single joint about z (gravity along z exerts no torque)
  has linear semi-implicit Euler dynamics, so with the quadratic joint cost one
  SQP step with alpha = 1 must reproduce the discrete Riccati solution.
* On the nonlinear arm, line-search invariants: every accepted step lowers the
  L1 merit, the KKT residual goes to zero, full steps are taken near the end.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I


def riccati_lqr(A, B, W, wr, WN, e0, N):
    P = WN.copy()
    Ks = []
    R = wr * np.eye(B.shape[1])
    for _ in range(N):
        K = np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
        P = W + A.T @ P @ A - A.T @ P @ B @ K
        Ks.append(K)
    Ks = Ks[::-1]
    e = e0.copy()
    E, Us = [e], []
    for k in range(N):
        u = -Ks[k] @ e
        e = A @ e + B @ u
        Us.append(u)
        E.append(e)
    return np.array(E), np.array(Us)


@pytest.mark.parametrize("N,h", [(5, 0.05), (20, 0.01)])
def test_one_sqp_step_equals_riccati_on_linear_joint(oracle, N, h):
    model = I.chain([2], [0.3], [1.0], name="1z")
    Izz = model.inertia[2]
    prob = I.joint_problem(3, model, N=N, dt=h)
    A = np.array([[1.0, h], [0.0, 1.0]])
    B = np.array([[h * h / Izz], [h / Izz]])
    wq, wqd, wr, ts = prob.w[:4]
    W = np.diag([wq, wqd])
    xr = prob.x_ref[0]
    E, Us = riccati_lqr(A, B, W, wr, ts * W, prob.x_s - xr, N)
    res = oracle.solve(prob, max_iter=1, replay=[0], pcg_eps=1e-13, pcg_max=10000)
    np.testing.assert_allclose(res["X"], E + xr, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(res["U"], Us, rtol=1e-9, atol=1e-9 * max(1, np.abs(Us).max()))
    # at the QP optimum of a linear-quadratic problem the KKT residual vanishes
    assert oracle.kkt_residual(prob, res["X"], res["U"], res["lam"]) < 1e-9
    # and the merit line search itself picks the full step
    free = oracle.solve(prob, max_iter=1, pcg_eps=1e-13, pcg_max=10000)
    assert free["alpha_idx"][0] == 0


def test_nonlinear_arm_invariants(oracle):
    prob = I.config_single()[0]
    res = oracle.solve(prob, max_iter=25)
    acc = res["alpha_idx"] >= 0
    assert acc.all()
    assert np.all(res["merit_after"] < res["merit_before"])
    assert res["kkt_log"][-1] < 1e-9
    # asymptotic regime, above the rounding floor: full steps are taken
    mid = (res["kkt_log"] < 1e-3) & (res["kkt_log"] > 1e-8)
    assert mid.sum() >= 5 and np.all(res["alpha_idx"][mid] == 0)
    # constraint violation of the final iterate is ~0 (dynamics satisfied)
    lin = oracle.linearize(prob, res["X"], res["U"])
    assert np.abs(lin["c"]).max() < 1e-7


def test_kkt_tolerance_stops_early(oracle):
    prob = I.config_single()[0]
    res = oracle.solve(prob, max_iter=40, kkt_tol=1e-5)
    assert res["flags"] & oracle.FLAG_CONVERGED
    assert res["kkt"] <= 1e-5
    assert res["iters"] < 40
    X, U = res["X"], res["U"]
    assert oracle.kkt_residual(prob, X, U, res["lam"]) <= 1e-5


def test_replay_reproduces_free_run(oracle):
    prob = I.joint_problem(11)
    free = oracle.solve(prob, max_iter=6)
    rep = oracle.solve(prob, max_iter=6, replay=free["alpha_idx"])
    np.testing.assert_array_equal(free["X"], rep["X"])
    np.testing.assert_array_equal(free["U"], rep["U"])


def test_cold_start_reading(oracle):
    prob = I.joint_problem(0)
    X, U, lam = oracle.cold_start(prob)
    assert np.all(X == prob.x_s) and np.all(U == 0) and np.all(lam == 0)


def test_merit_closed_form_at_cold_start(oracle):
    """Eq. 3 at X_k = x_s, U = 0: J has a closed form and c = [0, f(x_s,0) - x_s, ...]."""
    prob = I.joint_problem(4, I.arm7(), N=8, dt=0.01)
    X, U, _ = oracle.cold_start(prob)
    wq, wqd, wr, ts = prob.w[:4]
    W = np.diag([wq] * 7 + [wqd] * 7)
    d = prob.x_s - prob.x_ref[0]
    J = 0.5 * (prob.N + ts) * d @ W @ d
    e = oracle.step(prob.model, prob.x_s, np.zeros(7), prob.dt) - prob.x_s
    mu = 10.0
    want = J + mu * prob.N * np.abs(e).sum()
    assert abs(oracle.merit(prob, X, U, mu) - want) < 1e-12 * want
    pe = I.ee_problem(5, I.arm7(), N=6, dt=0.01)
    X, U, _ = oracle.cold_start(pe)
    wq, wqd, wr, ts, wee, rho = pe.w
    p = oracle.fk(pe.model, pe.x_s[:7])
    Jee = 0.5 * wee * (np.sum((p - pe.ee_ref[:-1]) ** 2) + ts * np.sum((p - pe.ee_ref[-1]) ** 2))
    e = oracle.step(pe.model, pe.x_s, np.zeros(7), pe.dt) - pe.x_s
    want = Jee + mu * pe.N * np.abs(e).sum()
    assert abs(oracle.merit(pe, X, U, mu) - want) < 1e-12 * want


def test_oracle_regression_fixture(oracle):
    """Record written by tests/golden/make_golden.py (oracle only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")
    with open(path) as f:
        gold = json.load(f)
    cases = {"config_single": I.config_single()[0],
             "arm6_seed1_N20": I.joint_problem(1, I.arm6(), N=20)}
    for key, prob in cases.items():
        g = gold[key]
        r = oracle.solve(prob, max_iter=g["iters"])
        assert r["alpha_idx"].tolist() == g["alpha_idx"]
        np.testing.assert_allclose(r["X"], np.array(g["X"]), atol=1e-9)
        np.testing.assert_allclose(r["U"], np.array(g["U"]), atol=1e-8)
        np.testing.assert_allclose(r["kkt_log"], g["kkt_log"], rtol=1e-8)


def test_direct_linear_solve_equals_converged_pcg(oracle):
    # The direct alternative to PCG (block elimination of S nu = rhs) and PCG
    # run to a tolerance far below FP64 noise solve the same QP each iteration,
    # so the SQP paths agree to rounding; the direct path takes no PCG steps.
    for p in (I.joint_problem(0, I.arm7(), 16, 0.01), I.ee_problem(2, I.arm7(), 12, 0.01)):
        a = oracle.solve(p, 3, pcg_eps=1e-12, pcg_max=5000)
        b = oracle.solve(p, 3, linsolve=1)
        assert b["pcg_total"] == 0 and b["flags"] == a["flags"]
        assert list(a["alpha_idx"]) == list(b["alpha_idx"])
        assert np.abs(a["X"] - b["X"]).max() <= 1e-9 * max(1.0, np.abs(a["X"]).max())
        assert np.abs(a["U"] - b["U"]).max() <= 1e-9 * max(1.0, np.abs(a["U"]).max())
        assert np.abs(a["lam"] - b["lam"]).max() <= 1e-7 * max(1.0, np.abs(a["lam"]).max())


def test_rho_adaptation_rule(oracle):
    # Sec. IV-C adjusts rho after each SQP iteration from the line search's
    # outcome (no factors given); here rho / 3 after an accepted step, rho * 2
    # after a rejected one, within the range [1e-8, 1e1] of Fig. 4.  The adapted run equals single
    # iterations with rho set by that rule between them.
    import dataclasses

    p0 = I.ee_problem(1, I.arm7(), 16, 0.05)
    p = dataclasses.replace(p0, w=tuple(p0.w[:5]) + (0.1,))
    full = oracle.solve(p, 8, rho_adapt=1)
    plain = oracle.solve(p, 8)
    assert np.abs(full["X"] - plain["X"]).max() > 1e-6  # the adaptation changes the path
    X, U, lam = oracle.cold_start(p)
    rho = 0.1
    for it in range(8):
        q = dataclasses.replace(p, w=tuple(p.w[:5]) + (rho,))
        r = oracle.solve(q, 1, X=X, U=U, lam=lam)
        assert r["alpha_idx"][0] == full["alpha_idx"][it]
        X, U, lam = r["X"], r["U"], r["lam"]
        rho = max(rho / 3.0, 1e-8) if r["alpha_idx"][0] >= 0 else min(rho * 2.0, 1e1)
    np.testing.assert_allclose(full["X"], X, rtol=0, atol=1e-12 * max(1.0, np.abs(X).max()))
    np.testing.assert_allclose(full["U"], U, rtol=0, atol=1e-12 * max(1.0, np.abs(U).max()))


def test_external_force_enters_defects_and_solution(oracle):
    """A solve with a constant end-effector force (Sec. IV-D's hypotheses):
    converged, its trajectory follows the forced dynamics (defects of the
    separately pinned one-step map with the force vanish) and not the free ones,
    and it differs from the unforced solve's."""
    import dataclasses

    base = I.joint_problem(3, I.arm6(), 16, 0.02)
    forced = dataclasses.replace(base, f_ext=(0.0, 0.0, -50.0))
    rf = oracle.solve(forced, max_iter=30, kkt_tol=1e-9)
    r0 = oracle.solve(base, max_iter=30, kkt_tol=1e-9)
    assert rf["flags"] & 1 and r0["flags"] & 1
    m, n = forced.model, forced.model.dof
    X, U = rf["X"].reshape(-1, 2 * n), rf["U"].reshape(-1, n)
    d_forced = max(np.abs(oracle.step(m, X[k], U[k], forced.dt, f_ext=forced.f_ext) - X[k + 1]).max()
                   for k in range(forced.N))
    d_free = max(np.abs(oracle.step(m, X[k], U[k], forced.dt) - X[k + 1]).max() for k in range(forced.N))
    assert d_forced < 1e-8
    assert d_free > 1e-3
    assert np.abs(rf["U"] - r0["U"]).max() > 1.0  # the controls push back against the force


@pytest.mark.parametrize("kind,model,seed,dt,warm,i_want", [
    ("joint", I.arm7(), 2, 0.05, 0, 3), ("joint", I.arm6(), 4, 0.05, 2, 2), ("joint", I.arm7(), 9, 0.02, 2, 0),
    ("ee", I.arm7(), 2, 0.05, 1, 2), ("ee", I.arm6(), 1, 0.05, 0, 3), ("ee_force", I.arm6(), 1, 0.05, 1, 4)],
    ids=["joint_arm7_cold_alpha1/8", "joint_arm6_alpha1/4", "joint_arm7_full_step", "ee_arm7_alpha1/4",
         "ee_arm6_cold_alpha1/8", "ee_force_arm6_alpha1/16"])
def test_one_nonlinear_sqp_iteration_from_pinned_parts(oracle, kind, model, seed, dt, warm, i_want):
    """One SQP iteration on the nonlinear arm rebuilt from separately pinned
    parts: the QP (Eq. 1) from the step Jacobians (pinned by central
    differences), the cost's gradient and (Gauss-Newton) Hessian written out
    from its definition (the end-effector terms through the FK Jacobian,
    pinned by a closed form and central differences; rho on the whole
    diagonal) and the one-step map's defects, solved densely in Eq. 1's
    convention; the merit (Eq. 3) by its definition at every alpha_i = 2^-i
    (Eq. 7); alpha* the first argmin.  The oracle's iteration must pick the
    same alpha and land on Z + alpha* dZ."""
    from tests.test_oracle_kkt import dense_kkt

    if kind == "ee_force":  # a constant end-effector force in the dynamics (Sec. IV-D)
        prob = I.disturbed_ee_problem(seed, (0.0, 0.0, -50.0), model, N=5, dt=dt)
    else:
        prob = (I.joint_problem if kind == "joint" else I.ee_problem)(seed, model, N=5, dt=dt)
    fe = np.array(prob.f_ext)
    n, N = model.dof, prob.N
    nx = 2 * n
    wq, wqd, wr, ts, wee, rho = prob.w
    W = np.diag([wq] * n + [wqd] * n)
    # the cold start or the iterate after `warm` oracle iterations
    if warm:
        rw = oracle.solve(prob, max_iter=warm, pcg_eps=1e-12, pcg_max=1000)
        X, U, lam = rw["X"].reshape(N + 1, nx), rw["U"].reshape(N, n), rw["lam"]
    else:
        X, U, lam = oracle.cold_start(prob)
        X, U = X.reshape(N + 1, nx), U.reshape(N, n)

    scale = [1.0] * N + [ts]

    def J(X, U):
        out = 0.5 * wr * np.sum(U ** 2)
        for k in range(N + 1):
            if kind == "joint":
                d = X[k] - prob.x_ref[k]
                out += 0.5 * scale[k] * d @ W @ d
            else:
                d = oracle.fk(model, X[k][:n]) - prob.ee_ref[k]
                out += 0.5 * scale[k] * (wee * d @ d + wqd * X[k][n:] @ X[k][n:])
        return out

    def expansion(k):
        """q_k and Q_k of the cost at X[k] (Gauss-Newton for the end effector)."""
        if kind == "joint":
            return scale[k] * W @ (X[k] - prob.x_ref[k]), scale[k] * W + rho * np.eye(nx)
        p, Jp = oracle.fk(model, X[k][:n], jacobian=True)
        q = np.concatenate([scale[k] * wee * Jp.T @ (p - prob.ee_ref[k]), scale[k] * wqd * X[k][n:]])
        Q = np.zeros((nx, nx))
        Q[:n, :n] = scale[k] * wee * Jp.T @ Jp
        Q[n:, n:] = scale[k] * wqd * np.eye(n)
        return q, Q + rho * np.eye(nx)

    def defects(X, U):
        c = [prob.x_s - X[0]] + [oracle.step(model, X[k], U[k], prob.dt, f_ext=fe) - X[k + 1] for k in range(N)]
        return np.array(c)

    def merit(X, U):
        return J(X, U) + 10.0 * np.abs(defects(X, U)).sum()

    AB = [oracle.step_jacobians(model, X[k], U[k], prob.dt, f_ext=fe) for k in range(N)]
    qQ = [expansion(k) for k in range(N + 1)]
    lin = dict(A=np.array([a for a, _ in AB]), B=np.array([b for _, b in AB]),
               Q=np.array([Q for _, Q in qQ]), R=np.array([wr * np.eye(n)] * N),
               q=np.array([q for q, _ in qQ]), r=wr * U, c=defects(X, U))
    G, g, C, c, xi, ui = dense_kkt(lin)
    nz, nc = G.shape[0], C.shape[0]
    K = np.block([[G, C.T], [C, np.zeros((nc, nc))]])
    dz = np.linalg.solve(K, np.concatenate([-g, c]))[:nz]
    dX = np.array([dz[xi(k):xi(k) + nx] for k in range(N + 1)])
    dU = np.array([dz[ui(k):ui(k) + n] for k in range(N)])
    m0 = merit(X, U)
    ms = [merit(X + 0.5 ** i * dX, U + 0.5 ** i * dU) for i in range(8)]
    i_star = int(np.argmin(ms))
    assert i_star == i_want  # the case exercises the step length it is meant to
    assert ms[i_star] < m0
    gap = sorted(ms)[1] - ms[i_star]
    assert gap > 1e-9 * m0  # not a near tie: the choice is unambiguous
    o = oracle.solve(prob, max_iter=1, X=X, U=U, lam=lam, pcg_eps=1e-12, pcg_max=1000)
    assert o["alpha_idx"][0] == i_star
    a = 0.5 ** i_star
    np.testing.assert_allclose(o["X"].reshape(N + 1, nx), X + a * dX, rtol=0, atol=1e-9)
    np.testing.assert_allclose(o["U"].reshape(N, n), U + a * dU, rtol=0, atol=1e-8)
    assert abs(o["merit_before"][0] - m0) <= 1e-10 * m0
    assert abs(o["merit_after"][0] - ms[i_star]) <= 1e-10 * m0
    # the KKT residual at this iterate with its multiplier, from the same pieces:
    # max(|c|_inf, |g + C^T nu|_inf / max(1, |g|_inf))
    nu = np.asarray(lam, dtype=np.float64).ravel()
    kkt = max(np.abs(c).max(), np.abs(g + C.T @ nu).max() / max(1.0, np.abs(g).max()))
    assert abs(oracle.kkt_residual(prob, X, U, lam) - kkt) <= 1e-12 * max(1.0, kkt)


def test_fixed_count_iterate_depends_on_pcg_truncation(oracle):
    """What a fixed-count comparison can ask of any implementation.

    Two FP64 runs of the method that differ only in how exactly each QP is
    solved (PCG stopped by its rule at eps = 1e-6, Sec. II-B, or the direct
    block elimination, its exact solution) follow the same step-length
    sequence, yet after the single-solve workload's 5 iterations from seed 5
    their iterates differ by more than 1e-4 relative: the unconverged SQP
    amplifies the PCG's per-step truncation (~1e-6 of the step).  Run to
    convergence, both reach the same KKT point.  So the iterate after a fixed
    count is determined by the method only up to this spread, and the GPU
    tests compare fixed-count iterates only where the spread is below 1e-5.
    """
    prob = I.joint_problem(5, I.arm7(), 32, 0.01)
    a = oracle.solve(prob, max_iter=5)
    b = oracle.solve(prob, max_iter=5, linsolve=1)
    assert list(a["alpha_idx"]) == list(b["alpha_idx"])
    rel = np.abs(a["X"] - b["X"]).max() / max(1.0, np.abs(b["X"]).max())
    assert rel > 1e-4, rel
    ca = oracle.solve(prob, max_iter=80, kkt_tol=1e-9)
    cb = oracle.solve(prob, max_iter=80, kkt_tol=1e-9, linsolve=1)
    assert ca["kkt"] <= 1e-7 and cb["kkt"] <= 1e-7
    np.testing.assert_allclose(ca["X"], cb["X"], atol=1e-6 * max(1.0, np.abs(cb["X"]).max()), rtol=0)
    # the same start at seed 1 is determined: there the spread is below 1e-5
    p1 = I.joint_problem(1, I.arm7(), 32, 0.01)
    a1 = oracle.solve(p1, max_iter=5)
    b1 = oracle.solve(p1, max_iter=5, linsolve=1)
    assert np.abs(a1["X"] - b1["X"]).max() / max(1.0, np.abs(b1["X"]).max()) < 1e-5
