"""Closed-loop disturbance rejection by hypothesize-and-test (Sec. IV-D).

A 6-DoF arm tracks the figure-eight with its end effector while an unmodelled
constant force pushes on the end effector.  Every control tick solves a batch
of M trajectory optimisations that differ only in the assumed force: the
current estimate and M-1 candidates around it (directions uniform on the
sphere, ``inputs.force_hypotheses``).  While the batch is being solved the
robot keeps moving under the previous control; when the solve returns, each
hypothesis' dynamics model predicts that motion from the tick's start state,
the hypothesis whose prediction is closest to the measured state is kept, its
first control is applied and the estimate is re-centred on its force.

The robot is the RK4 plant of the library (``gato.Plant``, 1 kHz, Sec. IV-E's
plant rate); the solve latency that the plant sees is the measured wall time
of the batch call (or a fixed value for reproducible runs), rounded up to
whole plant steps.  Larger batches sample the force more finely but take
longer per tick, which is the trade-off the case study measures.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I


@dataclass
class LoopResult:
    M: int
    ticks: int
    sim_s: float
    track_err_mean: float        # mean |p_ee - p_ref| (m) after the settling time
    track_err_max: float
    qd_abs_mean: float           # mean |qd| (rad/s) after the settling time
    solve_ms_mean: float
    solve_ms_p99: float
    f_est: tuple                 # force estimate at the end (N)
    f_err: float                 # |f_est - f_true| (N)
    picks: list = field(default_factory=list)  # chosen hypothesis index per tick


NONFINITE = 16  # the solve stopped on a non-finite value (gato_result.flags)


def select_hypothesis(plant, x_start, u_applied, steps, h, forces, x_measured, usable=None):
    """Index of the force whose model best predicts the measured state after
    ``steps`` plant steps from ``x_start`` under ``u_applied`` (ties: first),
    among the indices in ``usable`` (default: all); None if none is usable."""
    best, best_err = None, math.inf
    for j, f in enumerate(forces):
        if usable is not None and j not in usable:
            continue
        pred = plant.rk4(x_start, u_applied, h, steps, f_ext=f)
        err = float(np.linalg.norm(pred - x_measured))
        if err < best_err:
            best, best_err = j, err
    return best


class GpuBatchSolver:
    """Solves the tick's batch through the library (one gato_solve call;
    linsolve 1: the direct linear solve in place of PCG)."""

    def __init__(self, model, M, N, sqp_iters, stream=None, linsolve=0):
        from . import gato

        self.gato = gato
        self.B = gato.Batch([model], M, N, stream=stream, linsolve=linsolve)
        self.iters = sqp_iters

    def __call__(self, probs, X, U, lam, iters=None):
        hp = self.gato.HostProblems(self.B, probs, X=X, U=U, lam=lam)
        t0 = time.perf_counter()
        res = self.B.solve(hp.arr, hp.n, self.iters if iters is None else iters)
        dt = time.perf_counter() - t0
        out = self.gato.results_to_dicts(res, hp.n)
        return [dict(X=hp.X[i], U=hp.U[i], lam=hp.lam[i], **out[i]) for i in range(hp.n)], dt

    def close(self):
        self.B.close()


def run(solver, plant, M, f_true, *, model=None, N=32, dt=0.01, sim_s=1.0, plant_h=1e-3,
        radius=10.0, seed=0, settle_s=0.25, latency_s=None, warm_iters=20, f0=(0.0, 0.0, 0.0)):
    """One closed-loop run; ``solver(probs, X, U, lam, iters=None) ->
    (solutions, seconds)`` solves a batch (None: cold start; iters None: the
    solver's per-tick count).  ``latency_s``: None = the measured solve time,
    else this fixed time.  Before the first tick the estimate's problem is
    solved from the cold start with ``warm_iters`` iterations (untimed);
    ``f0`` is the initial force estimate.
    """
    model = model or plant.model
    base = I.ee_problem(seed, model, N, dt)
    t0 = base.meta["t0"]
    nq = model.dof
    x = np.asarray(base.x_s, dtype=np.float64).copy()
    f_hat = np.asarray(f0, dtype=np.float64).copy()
    f_true = np.asarray(f_true, dtype=np.float64)

    def problems(t, xs, forces):
        ref = I.figure_eight(t0 + t + dt * np.arange(N + 1))
        return [I.Problem(model, N, dt, xs.copy(), I.COST_EE, I.W_EE, ee_ref=ref, seed=seed,
                          f_ext=tuple(float(v) for v in f)) for f in forces]

    # initial trajectory: the estimate's problem solved from the cold start
    X = U = lam = None
    u_prev = np.zeros(nq)
    if warm_iters:
        sol0, _ = solver(problems(0.0, x, [f_hat]), None, None, None, iters=warm_iters)
        X, U, lam = [sol0[0]["X"]] * M, [sol0[0]["U"]] * M, [sol0[0]["lam"]] * M
        u_prev = np.array(sol0[0]["U"][0], dtype=np.float64)

    t = 0.0
    errs, qds, lat, picks = [], [], [], []
    tick = 0
    while t < sim_s:
        forces = I.force_hypotheses(seed * 100003 + tick, M, center=f_hat, radius=radius)
        sols, secs = solver(problems(t, x, forces), X, U, lam)
        secs = secs if latency_s is None else latency_s
        lat.append(secs)
        steps = max(1, int(math.ceil(secs / plant_h - 1e-9)))
        # the robot moves under the previous control while the batch is solved
        x_start = x.copy()
        for _ in range(steps):
            x = plant.rk4(x, u_prev, plant_h, 1, f_ext=f_true)
            t += plant_h
            if t >= settle_s:
                p = plant.ee(x[:nq])
                errs.append(float(np.linalg.norm(p - I.figure_eight(np.array([t0 + t]))[0])))
                qds.append(float(np.abs(x[nq:]).mean()))
        usable = {i for i, sl in enumerate(sols) if not (sl["flags"] & NONFINITE)}
        j = select_hypothesis(plant, x_start, u_prev, steps, plant_h, forces, x, usable)
        picks.append(j)
        if j is not None:  # else the previous control and warm start stay
            f_hat = np.asarray(forces[j], dtype=np.float64)
            u_prev = np.array(sols[j]["U"][0], dtype=np.float64)
            # every hypothesis warm-starts from the kept solution
            X = [sols[j]["X"]] * M
            U = [sols[j]["U"]] * M
            lam = [sols[j]["lam"]] * M
        tick += 1
    lat_ms = np.array(lat) * 1e3
    return LoopResult(M=M, ticks=tick, sim_s=t,
                      track_err_mean=float(np.mean(errs)) if errs else math.nan,
                      track_err_max=float(np.max(errs)) if errs else math.nan,
                      qd_abs_mean=float(np.mean(qds)) if qds else math.nan,
                      solve_ms_mean=float(lat_ms.mean()), solve_ms_p99=float(np.percentile(lat_ms, 99)),
                      f_est=tuple(float(v) for v in f_hat),
                      f_err=float(np.linalg.norm(f_hat - f_true)), picks=picks)
