"""Seeded synthetic workloads for the batched SQP solver.

This module only draws inputs: robot descriptions, start states, targets and
reference tracks, arrival times.  It holds none of the solver's arithmetic, so
both the FP64 oracle (through the tests) and the CUDA path are fed from here.

Workloads stand in for the paper's robots (6-DoF Indy7 in Sec. IV-B, 7-DoF
iiwa14 in Sec. IV-C/E), whose parameters are not published in the paper:

* ``arm7``: 7 revolute joints, axes z,y,z,y,z,y,z, links 0.2 m, 2.0 kg.
* ``arm6``: 6 revolute joints, axes z,y,z,y,z,y, links 0.25 m, 3.0 kg.

Link geometry: joint ``i`` sits at the parent joint's origin plus
``(0, 0, L)`` in the parent frame (joint 0 at the base origin), the link's
centre of mass is at ``(0, 0, L/2)`` in its own frame and the end effector at
``(0, 0, L)`` in the last frame.  Inertia about the centre of mass is that of
a rod of radius 0.05 m: ``diag(mL^2/12, mL^2/12, m r^2/2)`` (a zero axial
moment would make the mass matrix singular at q = 0).  Gravity is 9.81 m/s^2
along -z.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NQ_MAX = 7
NX_MAX = 14
NU_MAX = 7

AXIS_X, AXIS_Y, AXIS_Z = 0, 1, 2

COST_JOINT = 0
COST_EE = 1

ROD_RADIUS = 0.05
GRAVITY = 9.81

# Figure-eight end-effector track (Sec. IV-B task; amplitude and period from
# the benchmark configuration): p(t) = c + a * [0, sin wt, sin wt cos wt].
FIG8_CENTER = (0.5, 0.0, 0.7)
FIG8_AMPLITUDE = 0.15
FIG8_OMEGA = math.pi  # period 2 s

# Cost weights, in the order used everywhere: position, velocity, control,
# terminal scale, end-effector position, diagonal damping rho.
W_JOINT = (1.0, 0.1, 1e-3, 10.0, 0.0, 0.0)
# rho = 1 on the end-effector cost: with rho <= 1e-2 the Gauss-Newton Q_k (rank-3
# JᵀJ plus rho) makes FP32 PCG break down (Sec. IV-C uses rho as exactly this
# numerical-stability damping).
W_EE = (0.0, 0.1, 1e-3, 10.0, 100.0, 1.0)


@dataclass(frozen=True)
class ArmModel:
    """Serial revolute chain; arrays are padded to 7 joints."""

    dof: int
    axis: tuple
    link_len: tuple
    mass: tuple
    com: tuple  # dof*3, centre of mass in the link frame
    inertia: tuple  # dof*3, principal moments about the centre of mass
    gravity: float = GRAVITY
    name: str = ""

    @property
    def nx(self) -> int:
        return 2 * self.dof

    @property
    def nu(self) -> int:
        return self.dof


def _rod_arm(dof: int, axes, length: float, mass: float, name: str) -> ArmModel:
    ixx = mass * length * length / 12.0
    izz = mass * ROD_RADIUS * ROD_RADIUS / 2.0
    com, inertia = [], []
    for _ in range(dof):
        com += [0.0, 0.0, length / 2.0]
        inertia += [ixx, ixx, izz]
    return ArmModel(
        dof=dof,
        axis=tuple(axes[:dof]),
        link_len=tuple([length] * dof),
        mass=tuple([mass] * dof),
        com=tuple(com),
        inertia=tuple(inertia),
        name=name,
    )


def arm7() -> ArmModel:
    """7-DoF arm: axes z,y,z,y,z,y,z; links 0.2 m, 2.0 kg."""
    z, y = AXIS_Z, AXIS_Y
    return _rod_arm(7, (z, y, z, y, z, y, z), 0.2, 2.0, "arm7")


def arm6() -> ArmModel:
    """6-DoF variant: last joint dropped, links 0.25 m, 3.0 kg."""
    z, y = AXIS_Z, AXIS_Y
    return _rod_arm(6, (z, y, z, y, z, y), 0.25, 3.0, "arm6")


def chain(axes, lengths, masses, inertia_diag=None, com=None, name="chain") -> ArmModel:
    """Arbitrary small chain (used by the oracle pins on 1-2 link arms)."""
    dof = len(axes)
    if com is None:
        com = []
        for L in lengths:
            com += [0.0, 0.0, L / 2.0]
    if inertia_diag is None:
        inertia_diag = []
        for L, m in zip(lengths, masses):
            inertia_diag += [m * L * L / 12.0, m * L * L / 12.0, m * ROD_RADIUS**2 / 2.0]
    return ArmModel(dof, tuple(axes), tuple(lengths), tuple(masses), tuple(com),
                    tuple(inertia_diag), GRAVITY, name)


@dataclass
class Problem:
    """One trajectory-optimisation solve (Sec. II-A problem statement).

    ``x_ref`` is (N+1, nx) for the joint-space cost, ``ee_ref`` is (N+1, 3)
    for the end-effector cost; the unused one is None.
    """

    model: ArmModel
    N: int
    dt: float
    x_s: np.ndarray
    cost_kind: int
    w: tuple
    x_ref: np.ndarray | None = None
    ee_ref: np.ndarray | None = None
    seed: int = 0
    meta: dict = field(default_factory=dict)
    # constant external force on the end effector (base frame, N); Sec. IV-D's
    # disturbance hypotheses differ only in it
    f_ext: tuple = (0.0, 0.0, 0.0)


def figure_eight(t: np.ndarray) -> np.ndarray:
    """End-effector reference positions at times ``t`` (shape (len(t), 3))."""
    s = np.sin(FIG8_OMEGA * t)
    c = np.cos(FIG8_OMEGA * t)
    out = np.empty((len(t), 3))
    out[:, 0] = FIG8_CENTER[0]
    out[:, 1] = FIG8_CENTER[1] + FIG8_AMPLITUDE * s
    out[:, 2] = FIG8_CENTER[2] + FIG8_AMPLITUDE * s * c
    return out


def joint_problem(seed: int, model: ArmModel | None = None, N: int = 32,
                  dt: float = 0.01) -> Problem:
    """Reach a random joint target from a random start at rest.

    Draws, in order, from ``numpy.random.default_rng(seed)``:
    q_goal ~ U(-1, 1)^nq, then q0 ~ U(-1, 1)^nq; qd0 = 0.
    """
    model = model or arm7()
    rng = np.random.default_rng(seed)
    nq = model.dof
    q_goal = rng.uniform(-1.0, 1.0, nq)
    q0 = rng.uniform(-1.0, 1.0, nq)
    x_s = np.concatenate([q0, np.zeros(nq)])
    x_ref = np.tile(np.concatenate([q_goal, np.zeros(nq)]), (N + 1, 1))
    return Problem(model, N, dt, x_s, COST_JOINT, W_JOINT, x_ref=x_ref, seed=seed)


def ee_problem(seed: int, model: ArmModel | None = None, N: int = 64,
               dt: float = 0.01) -> Problem:
    """Track the figure-eight with the end effector.

    Draws q_goal (unused, kept so the first draws match ``joint_problem``),
    q0 ~ U(-1, 1)^nq, then the phase t0 ~ U(0, 2) s; knot k tracks
    p_ref(t0 + k dt).
    """
    model = model or arm7()
    rng = np.random.default_rng(seed)
    nq = model.dof
    rng.uniform(-1.0, 1.0, nq)
    q0 = rng.uniform(-1.0, 1.0, nq)
    t0 = rng.uniform(0.0, 2.0)
    x_s = np.concatenate([q0, np.zeros(nq)])
    ee_ref = figure_eight(t0 + dt * np.arange(N + 1))
    return Problem(model, N, dt, x_s, COST_EE, W_EE, ee_ref=ee_ref, seed=seed,
                   meta={"t0": t0})


def config_single(seed: int = 0) -> list[Problem]:
    """One joint-space solve, 7-DoF, N=32, dt=0.01 (5 SQP iterations)."""
    return [joint_problem(seed, arm7(), 32, 0.01)]


def config_fixed_batch(B: int = 32, N: int = 32) -> list[Problem]:
    """B joint-space solves with seeds 0..B-1, 7-DoF, dt=0.01 (10 iterations)."""
    return [joint_problem(b, arm7(), N, 0.01) for b in range(B)]


def config_sweep(B: int, N: int, seed0: int = 0) -> list[Problem]:
    """B figure-eight solves with seeds seed0..seed0+B-1, 7-DoF, horizon N, dt=0.01."""
    return [ee_problem(seed0 + b, arm7(), N, 0.01) for b in range(B)]


def uneven_horizon(seed: int) -> int:
    """Horizon of solve ``seed`` in the uneven mix: uniform on {16..128}."""
    return int(np.random.default_rng(seed).integers(16, 129))


def config_uneven(B: int = 128, seed0: int = 0) -> list[Problem]:
    """Uneven mix: solve b draws N_b ~ U{16..128} first, then q_goal and q0.

    Even b use the 7-DoF arm, odd b the 6-DoF arm.
    """
    out = []
    for i in range(B):
        b = seed0 + i
        rng = np.random.default_rng(b)
        N = int(rng.integers(16, 129))
        model = arm7() if b % 2 == 0 else arm6()
        nq = model.dof
        q_goal = rng.uniform(-1.0, 1.0, nq)
        q0 = rng.uniform(-1.0, 1.0, nq)
        x_s = np.concatenate([q0, np.zeros(nq)])
        x_ref = np.tile(np.concatenate([q_goal, np.zeros(nq)]), (N + 1, 1))
        out.append(Problem(model, N, 0.01, x_s, COST_JOINT, W_JOINT, x_ref=x_ref, seed=b))
    return out


def poisson_arrivals(rate: float, duration_s: float, n_clients: int,
                     seed: int = 12345, max_requests: int | None = None):
    """Arrival times (s) and client ids for the serving workload.

    Exponential inter-arrival gaps at ``rate`` requests/s; each arrival picks a
    client uniformly.  Draw order: all gaps, then all client ids.
    """
    rng = np.random.default_rng(seed)
    n_est = int(rate * duration_s * 1.2) + 16
    if max_requests is not None:
        n_est = min(n_est, max_requests)
    gaps = rng.exponential(1.0 / rate, n_est)
    t = np.cumsum(gaps)
    keep = t < duration_s
    t = t[keep]
    clients = rng.integers(0, n_clients, n_est)[keep]
    return t, clients


def state_disturbance(rng: np.random.Generator, nq: int, sigma_q: float = 0.05,
                      sigma_qd: float = 0.1) -> np.ndarray:
    """Gaussian disturbance added to the measured state between control ticks."""
    return np.concatenate([rng.normal(0.0, sigma_q, nq), rng.normal(0.0, sigma_qd, nq)])


def force_hypotheses(seed: int, M: int, center=(0.0, 0.0, 0.0), radius: float = 10.0) -> np.ndarray:
    """M candidate end-effector forces (N, base frame) around an estimate.

    Sec. IV-D samples directions uniformly on the sphere and adds them, scaled,
    to the current disturbance estimate.  Row 0 is the estimate itself; rows
    1..M-1 are ``center + radius * d`` with ``d`` a normalised standard-normal
    draw (uniform on the sphere).  Draws: an (M-1, 3) normal block.
    """
    rng = np.random.default_rng(seed)
    d = rng.normal(0.0, 1.0, (max(M - 1, 0), 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = np.empty((M, 3))
    out[0] = center
    out[1:] = np.asarray(center, dtype=float) + radius * d
    return out


def disturbed_ee_problem(seed: int, f_ext, model: ArmModel | None = None, N: int = 64,
                         dt: float = 0.01) -> Problem:
    """``ee_problem`` (figure-eight tracking) with a constant end-effector force."""
    p = ee_problem(seed, model, N, dt)
    p.f_ext = tuple(float(v) for v in f_ext)
    return p


def disturbed_joint_problem(seed: int, f_ext, model: ArmModel | None = None, N: int = 32,
                            dt: float = 0.01) -> Problem:
    """``joint_problem`` with a constant end-effector force."""
    p = joint_problem(seed, model, N, dt)
    p.f_ext = tuple(float(v) for v in f_ext)
    return p
