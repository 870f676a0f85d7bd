"""Pins for the oracle's rigid-body dynamics (the f(x, u, h) of Sec. II-A).

Nothing here re-types the oracle's formulas: the equations of motion come
from a symbolic Lagrangian (sympy), the derivatives from central differences,
the integrator from energy conservation and power balance, the kinematics
from a closed form.
"""
import numpy as np
import pytest
import sympy as sp

from paper_2510_07625_gb300 import inputs as I


def _rot(axis, q):
    c, s = sp.cos(q), sp.sin(q)
    if axis == 0:
        return sp.Matrix([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == 1:
        return sp.Matrix([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return sp.Matrix([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def lagrangian_eom(model):
    """tau(q, qd, qdd) from d/dt dL/dqd - dL/dq for a chain in the model's geometry."""
    n = model.dof
    t = sp.symbols("t")
    qf = [sp.Function(f"q{i}")(t) for i in range(n)]
    R = sp.eye(3)
    p = sp.zeros(3, 1)
    T = 0
    V = 0
    for i in range(n):
        if i > 0:
            p = p + R * sp.Matrix([0, 0, model.link_len[i - 1]])
        R = R * _rot(model.axis[i], qf[i])
        c = sp.Matrix(model.com[3 * i:3 * i + 3])
        pc = p + R * c
        vc = pc.diff(t)
        W = R.diff(t) * R.T
        w = sp.Matrix([W[2, 1], W[0, 2], W[1, 0]])
        Ib = sp.diag(*model.inertia[3 * i:3 * i + 3])
        T += sp.Rational(1, 2) * model.mass[i] * (vc.T * vc)[0] \
            + sp.Rational(1, 2) * (w.T * R * Ib * R.T * w)[0]
        V += model.mass[i] * model.gravity * pc[2]
    Lg = T - V
    qs = sp.symbols(f"q0:{n}")
    qds = sp.symbols(f"qd0:{n}")
    qdds = sp.symbols(f"qdd0:{n}")
    tau = []
    for j in range(n):
        e = sp.diff(sp.diff(Lg, qf[j].diff(t)), t) - sp.diff(Lg, qf[j])
        tau.append(e)
    subs = {}
    for j in range(n):
        subs[qf[j].diff(t, 2)] = qdds[j]
    for j in range(n):
        subs[qf[j].diff(t)] = qds[j]
    out = []
    for e in tau:
        e = e.subs(subs)
        e = e.subs({qf[j]: qs[j] for j in range(n)})
        out.append(e)
    return sp.lambdify((qs, qds, qdds), out, "numpy")


CHAINS = [
    I.chain([1], [0.3], [1.5], name="1y"),
    I.chain([0], [0.4], [2.0], name="1x"),
    I.chain([2, 1], [0.2, 0.3], [2.0, 1.0], name="2zy"),
    I.chain([1, 1], [0.25, 0.35], [1.0, 3.0], name="2yy"),
    I.chain([0, 2], [0.3, 0.2], [1.2, 0.8], inertia_diag=[0.01, 0.02, 0.03, 0.004, 0.005, 0.006],
            com=[0.01, -0.02, 0.12, 0.03, 0.0, 0.05], name="2xz_offset_com"),
]


@pytest.mark.parametrize("model", CHAINS, ids=lambda m: m.name)
def test_rnea_matches_lagrangian(oracle, model):
    f = lagrangian_eom(model)
    rng = np.random.default_rng(7)
    for _ in range(5):
        q, qd, qdd = (rng.uniform(-2, 2, model.dof) for _ in range(3))
        want = np.array(f(q, qd, qdd), dtype=float)
        got = oracle.rnea(model, q, qd, qdd)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("model", [I.arm7(), I.arm6()], ids=lambda m: m.name)
def test_mass_matrix_spd_and_inverse_dynamics_roundtrip(oracle, model):
    rng = np.random.default_rng(3)
    for _ in range(10):
        q, qd, tau = rng.uniform(-2, 2, model.dof), rng.uniform(-3, 3, model.dof), rng.uniform(-20, 20, model.dof)
        M = oracle.mass_matrix(model, q)
        np.testing.assert_allclose(M, M.T, atol=1e-14)
        assert np.linalg.eigvalsh(M).min() > 0
        qdd = oracle.forward_dynamics(model, q, qd, tau)
        np.testing.assert_allclose(oracle.rnea(model, q, qd, qdd), tau, rtol=1e-12, atol=1e-11)
        # M is the q̈-Jacobian of inverse dynamics: ID(q,qd,qdd) - ID(q,qd,0) = M qdd
        lin = oracle.rnea(model, q, qd, qdd) - oracle.rnea(model, q, qd, np.zeros(model.dof))
        np.testing.assert_allclose(lin, M @ qdd, rtol=1e-11, atol=1e-11)


def _fk_points(model, q):
    """Joint origins and link centres of mass in base coordinates (plain numpy)."""
    def rot(a, x):
        c, s = np.cos(x), np.sin(x)
        if a == 0:
            return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
        if a == 1:
            return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    R = np.eye(3)
    p = np.zeros(3)
    coms = []
    for i in range(model.dof):
        if i > 0:
            p = p + R @ np.array([0, 0, model.link_len[i - 1]])
        R = R @ rot(model.axis[i], q[i])
        coms.append(p + R @ np.array(model.com[3 * i:3 * i + 3]))
    ee = p + R @ np.array([0, 0, model.link_len[model.dof - 1]])
    return coms, ee


def _energy(oracle, model, x):
    n = model.dof
    q, qd = x[:n], x[n:]
    M = oracle.mass_matrix(model, q)
    coms, _ = _fk_points(model, q)
    V = sum(model.mass[i] * model.gravity * coms[i][2] for i in range(n))
    return 0.5 * qd @ M @ qd + V


def _rk4(oracle, model, x, tau, h):
    n = model.dof

    def f(y):
        return np.concatenate([y[n:], oracle.forward_dynamics(model, y[:n], y[n:], tau)])
    k1 = f(x)
    k2 = f(x + 0.5 * h * k1)
    k3 = f(x + 0.5 * h * k2)
    k4 = f(x + h * k3)
    return x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)


def test_energy_conservation_passive_arm(oracle):
    """tau = 0: RK4 at h = 1e-4 for 0.25 s keeps the total energy."""
    model = I.chain([2, 1, 1], [0.3, 0.3, 0.3], [2.0, 2.0, 2.0], name="3zyy")
    x = np.array([0.3, 0.6, -0.4, 1.0, 0.0, 0.5])
    E0 = _energy(oracle, model, x)
    scale = sum(model.mass) * model.gravity * sum(model.link_len)
    for _ in range(2500):
        x = _rk4(oracle, model, x, np.zeros(3), 1e-4)
    drift = abs(_energy(oracle, model, x) - E0) / scale
    assert drift < 1e-8


def test_power_balance(oracle):
    """dE/dt = qd^T tau along the exact flow (central difference of E)."""
    model = I.arm7()
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-1, 1, 7), rng.uniform(-1, 1, 7)])
    tau = rng.uniform(-5, 5, 7)
    h = 2e-6
    xp = _rk4(oracle, model, x, tau, h)
    xm = _rk4(oracle, model, x, tau, -h)
    dE = (_energy(oracle, model, xp) - _energy(oracle, model, xm)) / (2 * h)
    assert abs(dE - x[7:] @ tau) < 1e-6 * max(1.0, abs(x[7:] @ tau))


@pytest.mark.parametrize("model", [I.arm7(), I.arm6()], ids=lambda m: m.name)
def test_step_jacobians_match_central_differences(oracle, model):
    rng = np.random.default_rng(5)
    n = model.dof
    x = np.concatenate([rng.uniform(-1, 1, n), rng.uniform(-2, 2, n)])
    u = rng.uniform(-10, 10, n)
    h = 0.01
    A, B = oracle.step_jacobians(model, x, u, h)
    eps = 1e-6
    An = np.zeros_like(A)
    Bn = np.zeros_like(B)
    for j in range(2 * n):
        d = np.zeros(2 * n)
        d[j] = eps
        An[:, j] = (oracle.step(model, x + d, u, h) - oracle.step(model, x - d, u, h)) / (2 * eps)
    for j in range(n):
        d = np.zeros(n)
        d[j] = eps
        Bn[:, j] = (oracle.step(model, x, u + d, h) - oracle.step(model, x, u - d, h)) / (2 * eps)
    np.testing.assert_allclose(A, An, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(B, Bn, rtol=1e-6, atol=1e-8)


def test_semi_implicit_euler_structure(oracle):
    """q+ = q + h qd+, qd+ = qd + h qdd(q, qd, u)."""
    model = I.arm7()
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.uniform(-1, 1, 7), rng.uniform(-1, 1, 7)])
    u = rng.uniform(-5, 5, 7)
    h = 0.02
    qdd = oracle.forward_dynamics(model, x[:7], x[7:], u)
    xn = oracle.step(model, x, u, h)
    np.testing.assert_allclose(xn[7:], x[7:] + h * qdd, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(xn[:7], x[:7] + h * xn[7:], rtol=1e-14, atol=1e-14)


def test_fk_closed_form_planar_pair(oracle):
    model = I.chain([1, 1], [0.25, 0.35], [1.0, 1.0])
    for q1, q2 in [(0.0, 0.0), (0.3, -0.7), (1.2, 2.0)]:
        want = np.array([0.25 * np.sin(q1) + 0.35 * np.sin(q1 + q2), 0.0,
                         0.25 * np.cos(q1) + 0.35 * np.cos(q1 + q2)])
        np.testing.assert_allclose(oracle.fk(model, [q1, q2]), want, atol=1e-15)


def test_fk_jacobian_and_points(oracle):
    model = I.arm7()
    np.testing.assert_allclose(oracle.fk(model, np.zeros(7)), [0, 0, 1.4], atol=1e-15)
    rng = np.random.default_rng(2)
    q = rng.uniform(-1, 1, 7)
    p, J = oracle.fk(model, q, jacobian=True)
    _, ee = _fk_points(model, q)
    np.testing.assert_allclose(p, ee, atol=1e-14)
    eps = 1e-6
    for j in range(7):
        d = np.zeros(7)
        d[j] = eps
        col = (oracle.fk(model, q + d) - oracle.fk(model, q - d)) / (2 * eps)
        np.testing.assert_allclose(J[:, j], col, atol=1e-8)


# ------------------------------------------- external end-effector force
# Sec. IV-D's hypotheses differ only in a constant force on the end effector;
# the dynamics become M(q) qdd = tau + J_p(q)^T f - ID(q, qd, 0).

ARMS_AND_CHAINS = [I.arm7(), I.arm6()] + CHAINS


@pytest.mark.parametrize("model", ARMS_AND_CHAINS, ids=lambda m: m.name)
def test_ee_force_torque_is_fk_jacobian_transpose(oracle, model):
    """J_p^T f against the FK Jacobian (dual numbers through the FK chain) and
    against central differences of the FK position."""
    rng = np.random.default_rng(21)
    n = model.dof
    for _ in range(4):
        q = rng.uniform(-2, 2, n)
        f = rng.uniform(-50, 50, 3)
        _, J = oracle.fk(model, q, jacobian=True)
        np.testing.assert_allclose(oracle.ee_joint_torque(model, q, f), J.T @ f, rtol=1e-12, atol=1e-12)
        eps = 1e-6
        Jn = np.zeros((3, n))
        for j in range(n):
            d = np.zeros(n)
            d[j] = eps
            Jn[:, j] = (oracle.fk(model, q + d) - oracle.fk(model, q - d)) / (2 * eps)
        np.testing.assert_allclose(oracle.ee_joint_torque(model, q, f), Jn.T @ f, rtol=1e-7, atol=1e-7)


def _with_tip_mass(model, mp):
    """The same chain with a point mass mp added at the end-effector point."""
    n = model.dof
    L = model.link_len[n - 1]
    m0 = model.mass[n - 1]
    c0 = np.array(model.com[3 * (n - 1):3 * n])
    c1 = (m0 * c0 + mp * np.array([0.0, 0.0, L])) / (m0 + mp)
    mass = list(model.mass)
    mass[n - 1] = m0 + mp
    com = list(model.com)
    com[3 * (n - 1):3 * n] = list(c1)
    return I.ArmModel(n, model.axis, model.link_len, tuple(mass), tuple(com), model.inertia,
                      model.gravity, model.name + "_tipmass")


@pytest.mark.parametrize("model", [I.arm7(), I.arm6(), CHAINS[3]], ids=lambda m: m.name)
def test_ee_force_equals_tip_weight_in_statics(oracle, model):
    """At rest, a downward force m_p g on the end effector loads the joints like
    a point mass m_p there: the holding torques of the chain with the mass
    (inverse dynamics, gravity on) balance the chain without it plus the force,
    so its forward dynamics gives zero acceleration."""
    rng = np.random.default_rng(4)
    n = model.dof
    mp = 1.7
    heavy = _with_tip_mass(model, mp)
    f = np.array([0.0, 0.0, -mp * model.gravity])
    z = np.zeros(n)
    for _ in range(4):
        q = rng.uniform(-2, 2, n)
        hold = oracle.rnea(heavy, q, z, z)
        np.testing.assert_allclose(oracle.rnea(model, q, z, z) - oracle.ee_joint_torque(model, q, f), hold,
                                   rtol=1e-12, atol=1e-11)
        np.testing.assert_allclose(oracle.forward_dynamics(model, q, z, hold, f_ext=f), z, atol=1e-10)
        # without the force the same torques accelerate the arm
        assert np.abs(oracle.forward_dynamics(model, q, z, hold)).max() > 1e-3


def _rk4_force(oracle, model, x, tau, f, h):
    n = model.dof

    def fn(y):
        return np.concatenate([y[n:], oracle.forward_dynamics(model, y[:n], y[n:], tau, f_ext=f)])
    k1 = fn(x)
    k2 = fn(x + 0.5 * h * k1)
    k3 = fn(x + 0.5 * h * k2)
    k4 = fn(x + h * k3)
    return x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)


def test_energy_conservation_with_constant_ee_force(oracle):
    """A constant force is conservative with potential -f . p_ee: tau = 0, RK4
    at h = 1e-4 for 0.25 s keeps T + V_gravity - f . p_ee; the force's work is
    far above the drift bound."""
    model = I.chain([2, 1, 1], [0.3, 0.3, 0.3], [2.0, 2.0, 2.0], name="3zyy")
    f = np.array([12.0, -7.0, -30.0])
    x = np.array([0.3, 0.6, -0.4, 1.0, 0.0, 0.5])

    def energy(y):
        return _energy(oracle, model, y) - f @ oracle.fk(model, y[:3])
    E0 = energy(x)
    W0 = f @ oracle.fk(model, x[:3])
    scale = sum(model.mass) * model.gravity * sum(model.link_len)
    for _ in range(2500):
        x = _rk4_force(oracle, model, x, np.zeros(3), f, 1e-4)
    assert abs(energy(x) - E0) / scale < 1e-8
    assert abs(f @ oracle.fk(model, x[:3]) - W0) / scale > 1e-3


@pytest.mark.parametrize("model", [I.arm7(), I.arm6()], ids=lambda m: m.name)
def test_step_jacobians_with_ee_force_match_central_differences(oracle, model):
    rng = np.random.default_rng(15)
    n = model.dof
    x = np.concatenate([rng.uniform(-1, 1, n), rng.uniform(-2, 2, n)])
    u = rng.uniform(-10, 10, n)
    f = np.array([20.0, -10.0, -50.0])
    h = 0.01
    A, B = oracle.step_jacobians(model, x, u, h, f_ext=f)
    A0, _ = oracle.step_jacobians(model, x, u, h)
    eps = 1e-6
    An = np.zeros_like(A)
    Bn = np.zeros_like(B)
    for j in range(2 * n):
        d = np.zeros(2 * n)
        d[j] = eps
        An[:, j] = (oracle.step(model, x + d, u, h, f_ext=f) - oracle.step(model, x - d, u, h, f_ext=f)) / (2 * eps)
    for j in range(n):
        d = np.zeros(n)
        d[j] = eps
        Bn[:, j] = (oracle.step(model, x, u + d, h, f_ext=f) - oracle.step(model, x, u - d, h, f_ext=f)) / (2 * eps)
    np.testing.assert_allclose(A, An, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(B, Bn, rtol=1e-6, atol=1e-8)
    assert np.abs(A - A0).max() > 1e-4  # the force's q-dependence reaches A
