"""Pins for the oracle's QP / KKT / Schur / preconditioner / PCG (Eq. 1-6).

The references are textbook routines on dense matrices that the test builds
itself from the oracle's linearisation (A_k, B_k, Q_k, R_k, q_k, r_k, c):
numpy's dense LU for the full KKT system, dense C G^-1 C^T for the Schur
complement, dense inverses for the stair preconditioner identity.  The
linearisation itself is pinned in test_oracle_dynamics.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I


def dense_kkt(lin):
    """G, g, C, c of Eq. 2 with z = [x0, u0, x1, u1, ..., xN]."""
    A, B, Q, R, q, r, c = (lin[k] for k in "A B Q R q r c".split())
    N, nx, nu = B.shape
    nz = (N + 1) * nx + N * nu
    G = np.zeros((nz, nz))
    g = np.zeros(nz)
    C = np.zeros(((N + 1) * nx, nz))
    xi = lambda k: k * (nx + nu)
    ui = lambda k: k * (nx + nu) + nx
    for k in range(N + 1):
        G[xi(k):xi(k) + nx, xi(k):xi(k) + nx] = Q[k]
        g[xi(k):xi(k) + nx] = q[k]
        C[k * nx:(k + 1) * nx, xi(k):xi(k) + nx] = np.eye(nx)
        if k < N:
            G[ui(k):ui(k) + nu, ui(k):ui(k) + nu] = R[k]
            g[ui(k):ui(k) + nu] = r[k]
            C[(k + 1) * nx:(k + 2) * nx, xi(k):xi(k) + nx] = -A[k]
            C[(k + 1) * nx:(k + 2) * nx, ui(k):ui(k) + nu] = -B[k]
    return G, g, C, c.ravel(), xi, ui


def blocks_to_dense(Dd, Ls):
    N = Dd.shape[0] - 1
    nx = Dd.shape[1]
    M = np.zeros(((N + 1) * nx, (N + 1) * nx))
    for k in range(N + 1):
        M[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx] = Dd[k]
    for k in range(N):
        M[(k + 1) * nx:(k + 2) * nx, k * nx:(k + 1) * nx] = Ls[k]
        M[k * nx:(k + 1) * nx, (k + 1) * nx:(k + 2) * nx] = Ls[k].T
    return M


def _problems():
    small = I.chain([2, 1], [0.3, 0.3], [1.5, 1.0], name="2zy")
    p1 = I.joint_problem(4, small, N=3, dt=0.02)
    p2 = I.joint_problem(5, I.arm7(), N=4, dt=0.01)
    p3 = I.ee_problem(6, I.arm7(), N=3, dt=0.01)
    p4 = I.joint_problem(8, I.arm6(), N=2, dt=0.01)
    return [p1, p2, p3, p4]


def _midpoint(oracle, prob):
    """A non-trivial linearisation point: the iterate after one oracle SQP step."""
    r = oracle.solve(prob, max_iter=1)
    return r["X"], r["U"], r["lam"]


@pytest.mark.parametrize("prob", _problems(), ids=lambda p: f"{p.model.name}-N{p.N}-cost{p.cost_kind}")
def test_schur_blocks_equal_dense_CGinvCT(oracle, prob):
    X, U, _ = _midpoint(oracle, prob)
    lin = oracle.linearize(prob, X, U)
    G, g, C, c, _, _ = dense_kkt(lin)
    Gi = np.linalg.inv(G)
    S_dense = C @ Gi @ C.T
    rhs_dense = -c - C @ Gi @ g
    S = oracle.schur(prob, X, U)
    np.testing.assert_allclose(blocks_to_dense(S["Sd"], S["Ss"]), S_dense, rtol=1e-10,
                               atol=1e-10 * np.abs(S_dense).max())
    np.testing.assert_allclose(S["rhs"].ravel(), rhs_dense, rtol=1e-10,
                               atol=1e-10 * np.abs(rhs_dense).max())
    # S is block tridiagonal: nothing beyond the first off-diagonal block
    nx = S["Sd"].shape[1]
    for k in range(prob.N + 1):
        for l in range(prob.N + 1):
            if abs(k - l) > 1:
                assert np.abs(S_dense[k * nx:(k + 1) * nx, l * nx:(l + 1) * nx]).max() < 1e-14


@pytest.mark.parametrize("prob", _problems(), ids=lambda p: f"{p.model.name}-N{p.N}-cost{p.cost_kind}")
def test_qp_step_equals_dense_kkt_lu(oracle, prob):
    X, U, _ = _midpoint(oracle, prob)
    lin = oracle.linearize(prob, X, U)
    G, g, C, c, xi, ui = dense_kkt(lin)
    nz, m = G.shape[0], C.shape[0]
    K = np.block([[G, C.T], [C, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([-g, c]))
    dz = sol[:nz]
    # the convention of Eq. 1: C dZ = c, i.e. dx0 = x_s - x0, dx_{k+1} - A dx_k - B du_k = e_k
    np.testing.assert_allclose(C @ dz, c, atol=1e-10)
    dX, dU, nu, it = oracle.qp_step(prob, X, U, eps=1e-14, maxit=5000)
    nx, nu_ = lin["B"].shape[1], lin["B"].shape[2]
    for k in range(prob.N + 1):
        np.testing.assert_allclose(dX[k], dz[xi(k):xi(k) + nx], rtol=1e-9, atol=1e-9)
        if k < prob.N:
            np.testing.assert_allclose(dU[k], dz[ui(k):ui(k) + nu_], rtol=1e-9, atol=1e-8)
    np.testing.assert_allclose(nu.ravel(), sol[nz:], rtol=1e-8, atol=1e-8 * np.abs(sol[nz:]).max())


@pytest.mark.parametrize("prob", _problems(), ids=lambda p: f"{p.model.name}-N{p.N}-cost{p.cost_kind}")
def test_stair_preconditioner_identity_and_spd(oracle, prob):
    """Eq. 6 assembled from theta^-1 and phi equals D^-1 - D^-1 O D^-1 and is SPD."""
    X, U, _ = _midpoint(oracle, prob)
    S = oracle.schur(prob, X, U, precond=0)
    Sd = blocks_to_dense(S["Sd"], S["Ss"])
    nx = S["Sd"].shape[1]
    D = np.zeros_like(Sd)
    for k in range(prob.N + 1):
        D[k * nx:(k + 1) * nx, k * nx:(k + 1) * nx] = S["Sd"][k]
    O = Sd - D
    Di = np.linalg.inv(D)
    want = Di - Di @ O @ Di
    got = blocks_to_dense(S["Pd"], S["Ps"])
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    assert np.linalg.eigvalsh(0.5 * (got + got.T)).min() > 0
    # block Jacobi: diagonal blocks only
    J = oracle.schur(prob, X, U, precond=1)
    np.testing.assert_allclose(blocks_to_dense(J["Pd"], J["Ps"]), Di, rtol=1e-9,
                               atol=1e-9 * np.abs(Di).max())


def test_pcg_exact_preconditioner_one_iteration(oracle):
    """With Phi^-1 = S^-1 (N = 1, so S^-1 is block tridiagonal) PCG needs one iteration."""
    prob = I.joint_problem(1, I.arm7(), N=1, dt=0.01)
    X, U, _ = oracle.cold_start(prob)
    S = oracle.schur(prob, X, U)
    nx = 14
    Sinv = np.linalg.inv(blocks_to_dense(S["Sd"], S["Ss"]))
    Pd = np.stack([Sinv[:nx, :nx], Sinv[nx:, nx:]])
    Ps = Sinv[nx:, :nx][None]
    nu, it = oracle.pcg(S["Sd"], S["Ss"], Pd, Ps, S["rhs"], eps=1e-8, maxit=50)
    assert it == 1
    np.testing.assert_allclose(blocks_to_dense(S["Sd"], S["Ss"]) @ nu.ravel(), S["rhs"].ravel(),
                               rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("precond", [0, 1])
def test_pcg_and_block_cholesky_match_dense_solve(oracle, precond):
    prob = I.joint_problem(2, I.arm7(), N=12, dt=0.01)
    X, U, _ = oracle.cold_start(prob)
    S = oracle.schur(prob, X, U, precond=precond)
    Sd = blocks_to_dense(S["Sd"], S["Ss"])
    ref = np.linalg.solve(Sd, S["rhs"].ravel())
    direct = oracle.blocktri_solve(S["Sd"], S["Ss"], S["rhs"])
    np.testing.assert_allclose(direct.ravel(), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    nu, it = oracle.pcg(S["Sd"], S["Ss"], S["Pd"], S["Ps"], S["rhs"], eps=1e-13, maxit=20000)
    assert 1 < it < 20000
    np.testing.assert_allclose(nu.ravel(), ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


def test_pcg_stopping_rule(oracle):
    """Reading c8: stop when sqrt(eta / eta_0) <= eps, eta_0 from the warm start;
    no iteration at all when eta_0 < 1e-30."""
    prob = I.joint_problem(2, I.arm7(), N=6, dt=0.01)
    X, U, _ = oracle.cold_start(prob)
    S = oracle.schur(prob, X, U)
    nu, it = oracle.pcg(S["Sd"], S["Ss"], S["Pd"], S["Ps"], np.zeros_like(S["rhs"]), eps=1e-6,
                        maxit=100)
    assert it == 0 and np.all(nu == 0)
    exact = oracle.blocktri_solve(S["Sd"], S["Ss"], S["rhs"])
    for eps in (1e-3, 1e-6, 1e-9):
        nu, it = oracle.pcg(S["Sd"], S["Ss"], S["Pd"], S["Ps"], S["rhs"], eps=eps, maxit=5000)
        Sd = blocks_to_dense(S["Sd"], S["Ss"])
        Pm = blocks_to_dense(S["Pd"], S["Ps"])
        r = S["rhs"].ravel() - Sd @ nu.ravel()
        r0 = S["rhs"].ravel()
        # the recursively updated residual met the rule; the true one agrees to rounding
        assert np.sqrt((r @ Pm @ r) / (r0 @ Pm @ r0)) <= eps * 1.01 + 1e-10
    nu, it = oracle.pcg(S["Sd"], S["Ss"], S["Pd"], S["Ps"], S["rhs"], eps=1e-6, maxit=3)
    assert it == 3
    np.testing.assert_allclose(exact, oracle.blocktri_solve(S["Sd"], S["Ss"], S["rhs"]))


def test_stair_needs_fewer_iterations_than_jacobi(oracle):
    prob = I.joint_problem(0, I.arm7(), N=16, dt=0.01)
    X, U, _ = oracle.cold_start(prob)
    its = []
    for pc in (0, 1):
        S = oracle.schur(prob, X, U, precond=pc)
        its.append(oracle.pcg(S["Sd"], S["Ss"], S["Pd"], S["Ps"], S["rhs"], eps=1e-8, maxit=5000)[1])
    assert its[0] < its[1]


def test_fp32_storage_of_the_schur_matrix_moves_the_step(oracle):
    """The accuracy an FP32 step can have, measured with the oracle alone.

    At the cold start of a figure-eight solve (N = 64) the Schur complement
    S = C G^-1 C^T has a condition number near 1e9.  Rounding its assembled
    entries to FP32 and solving the residual-form system exactly in FP64
    changes the recovered step dZ = -G^-1 (d + C^T dnu) by 1e-4..2e-3 of its
    size, while rounding the inputs A, B, G^-1 it is formed from changes it by
    far less: an FP32 step is accurate to ~eps_32 sqrt(kappa(S)) of its size,
    whatever the solver.  (The GPU tests' per-step bound is this number.)
    """
    prob = I.ee_problem(1, I.arm7(), N=64, dt=0.01)
    X, U, lam = oracle.cold_start(prob)
    lin = oracle.linearize(prob, X, U)
    G, g, C, c, _, _ = dense_kkt(lin)
    Gi = np.linalg.inv(G)
    S = C @ Gi @ C.T
    d = g + C.T @ lam.ravel()
    rhs = -c - C @ Gi @ d
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    step = lambda Sm: -Gi @ (d + C.T @ np.linalg.solve(Sm, rhs))
    exact = step(S)
    moved = np.abs(step(f32(S)) - exact).max() / np.abs(exact).max()
    assert np.linalg.cond(S) > 1e8
    assert 1e-4 < moved < 2e-3, moved
    lin32 = {k: (f32(v) if isinstance(v, np.ndarray) else v) for k, v in lin.items()}
    G2, _, C2, _, _, _ = dense_kkt(lin32)
    S2 = C2 @ np.linalg.inv(G2) @ C2.T
    inputs_moved = np.abs(step(S2) - exact).max() / np.abs(exact).max()
    assert inputs_moved < 0.1 * moved, (inputs_moved, moved)
