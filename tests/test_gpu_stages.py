"""Stage-by-stage parity of the CUDA path against the FP64 oracle (Alg. 1 stages).

Each test runs the plain form of one solve through the C ABI up to a stage,
reads that solve's workspace back, and compares the stage's output with the
oracle's same quantity on the same inputs.  Tolerances are FP32 ones: the
dynamics Jacobians go through M^-1 (condition ~1e3), so they get 1e-4
relative to the block's largest entry; pure recombinations (recovery, merit)
of GPU-produced data are checked against the oracle's formula applied to
that data, in FP64, at 1e-5.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I

pytestmark = pytest.mark.gpu

VS, US, BS, XM = 16, 8, 199, 14


def pad_idx(dof):
    return list(range(dof)) + [7 + i for i in range(dof)]


@pytest.fixture(scope="module")
def G():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07625_gb300 import build, gato

    build.build_library()
    gato.load()
    return gato


def stage(G, prob, st, X=None, U=None, lam=None, **prm):
    B = G.Batch([prob.model], 1, prob.N, **prm)
    hp = G.HostProblems(B, [prob],
                        X=None if X is None else [X.astype(np.float32)],
                        U=None if U is None else [U.astype(np.float32)],
                        lam=None if lam is None else [lam.astype(np.float32)])
    buf, off = G.gato_debug_plain_stage(B.handle, hp.arr, st)
    total, _ = G.gato_debug_layout(B.handle)
    B.close()
    return buf.astype(np.float64), off, prob.N


def knots(buf, off, name, K, stride, n):
    return buf[off[name]:off[name] + K * stride].reshape(K, stride)[:, :n]


def block(buf, off, name, K):
    a = buf[off[name]:off[name] + K * BS].reshape(K, BS)[:, :196].reshape(K, XM, XM)
    return np.transpose(a, (0, 2, 1))  # stored column-major


# vector slots of the plain form's global window (one halo knot at each end)
V_RR, V_P0, V_P1, V_Q, V_Y, V_W, V_Z, V_RHS, V_DNU = range(9)


VW = 18  # knot stride of the vector windows


def vec(buf, off, k_max, idx):
    VV = (k_max + 3) * VW
    base = off["vec"] + idx * VV + VW
    return buf[base:base + (k_max + 1) * VW].reshape(k_max + 1, VW)[:, :XM]


PROBS = [
    ("arm7_joint", lambda: I.joint_problem(0, I.arm7(), N=8, dt=0.01)),
    ("arm6_joint", lambda: I.joint_problem(3, I.arm6(), N=6, dt=0.02)),
    ("arm7_ee", lambda: I.ee_problem(2, I.arm7(), N=7, dt=0.01)),
    # a constant end-effector force (Sec. IV-D): in the bias, the tangents and
    # the line search's dynamics
    ("arm6_ee_force", lambda: I.disturbed_ee_problem(5, (0.0, 0.0, -50.0), I.arm6(), N=7, dt=0.01)),
    ("arm7_joint_force", lambda: I.disturbed_joint_problem(1, (20.0, -10.0, -30.0), I.arm7(), N=8, dt=0.01)),
]


def lam_padded(lam, pi, K):
    out = np.zeros((K, XM))
    out[:, pi] = lam
    return out


def midpoint(oracle, prob):
    r = oracle.solve(prob, max_iter=2)
    return r["X"], r["U"], r["lam"]


@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_linearisation_stage(G, oracle, name, mk):
    prob = mk()
    X, U, lam = midpoint(oracle, prob)
    buf, off, N = stage(G, prob, 6, X, U, lam)
    K = N + 1
    dof = prob.model.dof
    pi = pad_idx(dof)
    lin = oracle.linearize(prob, X, U)
    h = prob.dt
    Fq = buf[off["Fq"]:off["Fq"] + N * 49].reshape(N, 7, 7)
    Fv = buf[off["Fv"]:off["Fv"] + N * 49].reshape(N, 7, 7)
    Mi = buf[off["Minv"]:off["Minv"] + N * 49].reshape(N, 7, 7)
    I7 = np.eye(7)
    for k in range(N):
        A = np.block([[I7 + h * h * Fq[k], h * I7 + h * h * Fv[k]], [h * Fq[k], I7 + h * Fv[k]]])
        Bm = np.vstack([h * h * Mi[k], h * Mi[k]])
        A = A[np.ix_(pi, pi)]
        Bm = Bm[np.ix_(pi, list(range(dof)))]
        sA = np.abs(lin["A"][k]).max()
        sB = np.abs(lin["B"][k]).max()
        np.testing.assert_allclose(A, lin["A"][k], atol=1e-4 * sA, rtol=0)
        np.testing.assert_allclose(Bm, lin["B"][k], atol=1e-4 * sB, rtol=0)
    c = knots(buf, off, "c", K, VS, XM)[:, pi]
    np.testing.assert_allclose(c, lin["c"], atol=2e-5 * max(1, np.abs(X).max()), rtol=0)
    q = knots(buf, off, "q", K, VS, XM)[:, pi]
    np.testing.assert_allclose(q, lin["q"], atol=1e-4 * max(1, np.abs(lin["q"]).max()), rtol=0)
    r = knots(buf, off, "r", N, US, dof)
    np.testing.assert_allclose(r, lin["r"], atol=1e-5 * max(1, np.abs(lin["r"]).max()), rtol=0)
    Qi = buf[off["Qinv"]:off["Qinv"] + K * 56].reshape(K, 56)
    for k in range(K):
        Qfull = np.zeros((14, 14))
        Qfull[:7, :7] = Qi[k, :49].reshape(7, 7)
        Qfull[7:, 7:] = np.diag(Qi[k, 49:56])
        want = np.linalg.inv(lin["Q"][k])
        np.testing.assert_allclose(Qfull[np.ix_(pi, pi)], want, atol=2e-4 * np.abs(want).max(), rtol=0)
    # dual residual d = g + C^T nu (compensated on the GPU) against the oracle in FP64
    t = lin["q"] + lam
    t[:-1] -= np.einsum("kji,kj->ki", lin["A"], lam[1:])
    du_want = lin["r"] - np.einsum("kji,kj->ki", lin["B"], lam[1:])
    Dx = knots(buf, off, "Dx", K, VS, XM)[:, pi]
    Du = knots(buf, off, "Du", N, US, dof)
    scale = max(1.0, np.abs(lin["q"]).max(), np.abs(lam).max())
    np.testing.assert_allclose(Dx, t, atol=1e-4 * scale, rtol=0)
    np.testing.assert_allclose(Du, du_want, atol=1e-4 * scale, rtol=0)
    # KKT residual and merit of the current iterate, against the oracle (FP64)
    scal = buf[off["scal"]:off["scal"] + 64]
    kkt_ora = oracle.kkt_residual(prob, X, U, lam)
    assert abs(scal[0] - kkt_ora) <= 1e-4 * max(1.0, kkt_ora)
    m_ora = oracle.merit(prob, X, U)
    assert abs(scal[1] - m_ora) <= 1e-5 * m_ora


@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_schur_and_preconditioner_stage(G, oracle, name, mk):
    prob = mk()
    X, U, lam = midpoint(oracle, prob)
    buf, off, N = stage(G, prob, 8, X, U, lam)
    K = N + 1
    h = prob.dt
    pi = pad_idx(prob.model.dof)
    S = oracle.schur(prob, X, U)
    D = block(buf, off, "D", K)
    L = block(buf, off, "L", K)
    P = block(buf, off, "P", K)
    rhs = vec(buf, off, prob.N, V_RHS)
    # (1) the stage's own arithmetic: Eq. 5 blocks and the correction rhs
    #     recomputed in FP64 from the GPU's inputs to this stage
    Fq = buf[off["Fq"]:off["Fq"] + N * 49].reshape(N, 7, 7)
    Fv = buf[off["Fv"]:off["Fv"] + N * 49].reshape(N, 7, 7)
    Mi = buf[off["Minv"]:off["Minv"] + N * 49].reshape(N, 7, 7)
    Qi = buf[off["Qinv"]:off["Qinv"] + K * 56].reshape(K, 56)
    Ri = knots(buf, off, "Rinv", N, US, 7)
    Dx = knots(buf, off, "Dx", K, VS, XM)
    Du = knots(buf, off, "Du", N, US, 7)
    cv = knots(buf, off, "c", K, VS, XM)
    I7 = np.eye(7)
    Qf = np.zeros((K, 14, 14))
    for k in range(K):
        Qf[k, :7, :7] = Qi[k, :49].reshape(7, 7)
        Qf[k, 7:, 7:] = np.diag(Qi[k, 49:])
    D_want = [Qf[0]]
    L_want = [np.zeros((14, 14))]
    rhs_want = [-cv[0] - Qf[0] @ Dx[0]]
    for k in range(N):
        A = np.block([[I7 + h * h * Fq[k], h * I7 + h * h * Fv[k]], [h * Fq[k], I7 + h * Fv[k]]])
        Bm = np.vstack([h * h * Mi[k], h * Mi[k]])
        BRB = Bm @ np.diag(Ri[k]) @ Bm.T
        Lk = -A @ Qf[k]
        D_want.append(A @ Qf[k] @ A.T + BRB + Qf[k + 1])
        L_want.append(Lk)
        zeta = Lk @ Dx[k] - Bm @ np.diag(Ri[k]) @ Du[k] + Qf[k + 1] @ Dx[k + 1]
        rhs_want.append(-cv[k + 1] - zeta)
    for k in range(K):
        sc = np.abs(D_want[k]).max()
        np.testing.assert_allclose(D[k], D_want[k], atol=2e-6 * sc, rtol=0)
        if k > 0:
            np.testing.assert_allclose(L[k], L_want[k], atol=2e-6 * np.abs(L_want[k]).max(), rtol=0)
    rw = np.array(rhs_want)
    np.testing.assert_allclose(rhs, rw, atol=1e-5 * max(1e-6, np.abs(rw).max()), rtol=0)
    # (2) the blocks against the oracle's Schur complement (FP32 Jacobians)
    for k in range(K):
        Dk = D[k][np.ix_(pi, pi)]
        np.testing.assert_allclose(Dk, S["Sd"][k], atol=1e-4 * np.abs(S["Sd"][k]).max(), rtol=0)
        # the GPU's D^-1 inverts the GPU's own D to FP32 working accuracy
        Pg = P[k][np.ix_(pi, pi)]
        kappa = np.linalg.cond(Dk)
        assert np.abs(Pg @ Dk - np.eye(len(pi))).max() < 50 * kappa * 6e-8
        if k > 0:
            Lk = L[k][np.ix_(pi, pi)]
            np.testing.assert_allclose(Lk, S["Ss"][k - 1], atol=1e-4 * np.abs(S["Ss"][k - 1]).max(), rtol=0)


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_pcg_recovery_and_line_search_stages(G, oracle, name, mk, precond):
    prob = mk()
    X, U, lam = midpoint(oracle, prob)
    N, K = prob.N, prob.N + 1
    dof = prob.model.dof
    pi = pad_idx(dof)
    buf, off, _ = stage(G, prob, 11, X, U, lam, precond=precond)
    # PCG on the GPU's own Schur system (read back, evaluated in FP64): the
    # multiplier meets the relative stopping rule up to FP32 attainable accuracy
    D = block(buf, off, "D", K)
    L = block(buf, off, "L", K)
    P = block(buf, off, "P", K)
    rhs_g = vec(buf, off, N, V_RHS)
    nu_g = knots(buf, off, "nu", K, VS, XM)
    from tests.test_oracle_kkt import blocks_to_dense
    Sg = blocks_to_dense(D, L[1:])
    Dinv = np.zeros_like(Sg)
    for k in range(K):
        Dinv[k * XM:(k + 1) * XM, k * XM:(k + 1) * XM] = P[k]
    Og = Sg.copy()
    for k in range(K):
        Og[k * XM:(k + 1) * XM, k * XM:(k + 1) * XM] = 0
    Phi = Dinv - Dinv @ Og @ Dinv if precond == 0 else Dinv
    dnu = vec(buf, off, N, V_DNU)
    r0 = rhs_g.ravel()
    r = rhs_g.ravel() - Sg @ dnu.ravel()
    nu_g = dnu
    rel = np.sqrt(abs(r @ Phi @ r) / (r0 @ Phi @ r0))
    exact = np.linalg.solve(Sg, rhs_g.ravel())
    assert rel < 1e-4, rel
    # the error in the S-norm (the step's error in the G-norm: dZ changes by
    # G^-1 C^T e, and |G^-1 C^T e|_G^2 = e^T S e).  In exact arithmetic the
    # stopping rule bounds it by eps sqrt(kappa(Phi S)); FP32 adds its
    # attainable accuracy ~eps_32 sqrt(kappa(S)), with a factor 10 for the
    # iteration's accumulated rounding
    e = nu_g.ravel() - exact
    err_S = np.sqrt(abs(e @ Sg @ e) / (exact @ Sg @ exact))
    ev = np.linalg.eigvalsh(Sg)
    kappa_S = ev.max() / ev.min()
    evp = np.linalg.eigvals(Phi @ Sg).real
    kappa_PS = evp.max() / evp.min()
    bound = 1e-6 * np.sqrt(kappa_PS) + 10 * 6e-8 * np.sqrt(kappa_S)
    assert err_S <= bound, (err_S, bound, kappa_S, kappa_PS)
    # recovery: dZ = -G^-1 (g + C^T nu) on the GPU's own linearisation and nu, in FP64
    h = prob.dt
    Fq = buf[off["Fq"]:off["Fq"] + N * 49].reshape(N, 7, 7)
    Fv = buf[off["Fv"]:off["Fv"] + N * 49].reshape(N, 7, 7)
    Mi = buf[off["Minv"]:off["Minv"] + N * 49].reshape(N, 7, 7)
    Qi = buf[off["Qinv"]:off["Qinv"] + K * 56].reshape(K, 56)
    Ri = knots(buf, off, "Rinv", N, US, 7)
    qg = knots(buf, off, "q", K, VS, XM)
    rg = knots(buf, off, "r", N, US, 7)
    nup = vec(buf, off, N, V_DNU)
    Dx = knots(buf, off, "Dx", K, VS, XM)
    Du = knots(buf, off, "Du", N, US, 7)
    I7 = np.eye(7)
    dX_want = np.zeros((K, XM))
    dU_want = np.zeros((N, 7))
    cancel = 0.0
    for k in range(K):
        t = Dx[k] + nup[k]
        if k < N:
            A = np.block([[I7 + h * h * Fq[k], h * I7 + h * h * Fv[k]], [h * Fq[k], I7 + h * Fv[k]]])
            Bm = np.vstack([h * h * Mi[k], h * Mi[k]])
            t = t - A.T @ nup[k + 1]
            dU_want[k] = -Ri[k] * (Du[k] - Bm.T @ nup[k + 1])
            # FP32 rounding of the two terms before R^-1 (= 1e3) scales them up
            cancel = max(cancel, np.abs(Ri[k]).max() * max(np.abs(Du[k]).max(), np.abs(Bm.T @ nup[k + 1]).max()))
        Qf = np.zeros((14, 14))
        Qf[:7, :7] = Qi[k, :49].reshape(7, 7)
        Qf[7:, 7:] = np.diag(Qi[k, 49:])
        dX_want[k] = -Qf @ t
    dX = knots(buf, off, "dX", K, VS, XM)
    dU = knots(buf, off, "dU", N, US, 7)
    np.testing.assert_allclose(dX, dX_want, atol=1e-5 * np.abs(dX_want).max(), rtol=0)
    np.testing.assert_allclose(dU, dU_want, atol=1e-5 * np.abs(dU_want).max() + 8 * 6e-8 * cancel, rtol=0)
    dX, dU = dX[:, pi], dU[:, :dof]
    # line search: trial merits of the GPU step, against the oracle merit in FP64
    scal = buf[off["scal"]:off["scal"] + 64]
    for a in range(8):
        al = 0.5 ** a
        m_ora = oracle.merit(prob, X + al * dX, U + al * dU)
        assert abs(scal[16 + a] - m_ora) <= 2e-5 * m_ora, (a, scal[16 + a], m_ora)


EPS32 = 2.0 ** -24


def f32_problem(prob):
    """The problem as the GPU holds it: model parameters, gravity, time step,
    force, initial state, cost weights and references rounded to float32
    (the oracle then evaluates the same problem, so only the arithmetic
    differs)."""
    import dataclasses

    r = lambda t: tuple(float(np.float32(v)) for v in t)
    a = lambda x: None if x is None else np.asarray(x, np.float32).astype(np.float64)
    m = prob.model
    fm = dataclasses.replace(m, link_len=r(m.link_len), mass=r(m.mass), com=r(m.com), inertia=r(m.inertia),
                             gravity=float(np.float32(m.gravity)))
    return dataclasses.replace(prob, model=fm, dt=float(np.float32(prob.dt)), f_ext=r(prob.f_ext),
                               x_s=a(prob.x_s), w=r(prob.w), x_ref=a(prob.x_ref), ee_ref=a(prob.ee_ref))


@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_high_precision_dynamics_stages(G, oracle, name, mk):
    """The high-precision mode's dynamics (GATO_PRECISION_HIGH, plain form)
    against the FP64 oracle on the float32-rounded model.  After the mass
    stage M and the bias
    ID(q, qd, 0) - J_p^T f_ext, kept as (hi, lo) float pairs, carry the
    double-float accuracy of their arithmetic (1e-10 of their scale here; the
    FP32 mode's error is ~1e-6).  After the forward dynamics the stored qdd
    is refined once with the FP32 factor: error ~(kappa(M) eps_32)^2 from the
    refinement plus its FP32 rounding, and the defects carry h times that
    plus their own rounding."""
    prob = mk()
    X, U, lam = midpoint(oracle, prob)
    N, K = prob.N, prob.N + 1
    dof = prob.model.dof
    Xf = X.astype(np.float32).astype(np.float64)
    Uf = U.astype(np.float32).astype(np.float64)
    buf, off, _ = stage(G, prob, 1, X, U, lam, precision=2)
    prob = f32_problem(prob)
    f = np.array(prob.f_ext, dtype=np.float64)
    DTS = 112
    for k in range(N):
        q, qd = Xf[k, :dof], Xf[k, dof:]
        M_ora = oracle.mass_matrix(prob.model, q)
        b_ora = oracle.rnea(prob.model, q, qd, np.zeros(dof)) - oracle.ee_joint_torque(prob.model, q, f)
        hi = buf[off["Minv"] + k * 49:off["Minv"] + k * 49 + 49].reshape(7, 7)
        lo = buf[off["dTau"] + k * DTS:off["dTau"] + k * DTS + 56].reshape(7, 8)[:, :7].T  # lo[r][col] at col * 8 + r
        M_gpu = (hi + lo)[:dof, :dof]
        np.testing.assert_allclose(M_gpu, M_ora, atol=1e-10 * max(1.0, np.abs(M_ora).max()), rtol=0)
        b_gpu = buf[off["qdd"] + k * US:off["qdd"] + k * US + dof] + \
            buf[off["dTau"] + k * DTS + 56:off["dTau"] + k * DTS + 56 + dof]
        np.testing.assert_allclose(b_gpu, b_ora, atol=1e-10 * max(1.0, np.abs(b_ora).max()), rtol=0)
    buf, off, _ = stage(G, prob, 2, X, U, lam, precision=2)
    qdd_gpu = knots(buf, off, "qdd", N, US, dof)
    qdd_ora = np.array([oracle.forward_dynamics(prob.model, Xf[k, :dof], Xf[k, dof:], Uf[k], f) for k in range(N)])
    kappa = max(np.linalg.cond(oracle.mass_matrix(prob.model, Xf[k, :dof])) for k in range(N))
    tol_qdd = np.abs(qdd_ora).max() * (10 * (kappa * EPS32) ** 2 + 4 * EPS32)
    np.testing.assert_allclose(qdd_gpu, qdd_ora, atol=tol_qdd, rtol=0)
    lin = oracle.linearize(prob, Xf, Uf)
    c = knots(buf, off, "c", K, VS, XM)[:, pad_idx(dof)]
    tol_c = prob.dt * tol_qdd + 4 * EPS32 * max(1.0, np.abs(lin["c"]).max())
    np.testing.assert_allclose(c, lin["c"], atol=tol_c, rtol=0)


@pytest.mark.parametrize("name,mk", PROBS, ids=[p[0] for p in PROBS])
def test_high_precision_line_search_stage(G, oracle, name, mk):
    """The high-precision mode's trial merits (double-float pairs) against the
    oracle's merit on the float32-rounded problem at the same trial points:
    with a zero low part the trial point X + alpha dX is exact on both sides,
    and qdd, refined twice, errs by ~(kappa(M) eps_32)^3, so the merits agree
    to 1e-9 relative (the FP32 mode's bound is 2e-5)."""
    prob = mk()
    X, U, lam = midpoint(oracle, prob)
    N, K = prob.N, prob.N + 1
    dof = prob.model.dof
    pi = pad_idx(dof)
    buf, off, _ = stage(G, prob, 11, X, U, lam, precision=2)
    pf = f32_problem(prob)
    Xf = X.astype(np.float32).astype(np.float64)
    Uf = U.astype(np.float32).astype(np.float64)
    dX = knots(buf, off, "dX", K, VS, XM)[:, pi]
    dU = knots(buf, off, "dU", N, US, 7)[:, :dof]
    scal = buf[off["scal"]:off["scal"] + 128]
    for a in range(8):
        al = 0.5 ** a
        m_gpu = scal[66 + 2 * a] + scal[67 + 2 * a]
        m_ora = oracle.merit(pf, Xf + al * dX, Uf + al * dU)
        assert abs(m_gpu - m_ora) <= 1e-9 * m_ora, (a, m_gpu, m_ora)

