"""Serving loop (continuous batching of MPC control ticks) on the GPU.

A request's arithmetic depends only on its own session and its cluster size
(fixed by the horizon), so a tick must give the same bits alone, in any mix,
and as the equivalent gato_solve call.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I
from tests.test_gpu_parity import gpu_solve

pytestmark = pytest.mark.gpu

MODELS = [I.arm7(), I.arm6()]


@pytest.fixture(scope="module")
def S():
    from paper_2510_07625_gb300 import gato, serving
    gato.load()
    return serving


def _mix(n=12):
    return I.config_uneven(B=n)


@pytest.mark.parametrize("linsolve", [0, 1], ids=["pcg", "direct"])
def test_tick_equals_gato_solve(S, linsolve):
    probs = _mix(4)
    # sessions carry the end-effector force (Sec. IV-D) like gato_solve's problems
    probs[1].f_ext = (10.0, -5.0, -40.0)
    srv = S.Server(MODELS, 8, 128, sqp_iters=3, linsolve=linsolve)
    for p in probs:
        sid = srv.open(p)
        r = srv.tick(sid, p.x_s, shift=False)
        X, U, lam = srv.read(sid)
        g = gpu_solve(S.gato, [p], 3, linsolve=linsolve)[0]
        np.testing.assert_array_equal(X, g["X"].astype(np.float32))
        np.testing.assert_array_equal(U, g["U"].astype(np.float32))
        np.testing.assert_array_equal(lam, g["lam"].astype(np.float32))
        assert (r.result.flags, r.result.sqp_iters, r.result.pcg_iters) == (g["flags"], g["sqp_iters"], g["pcg_iters"])
        np.testing.assert_array_equal(np.array(r.u0[:p.model.dof], np.float32), U[0])
        np.testing.assert_array_equal(np.array(r.x1[:2 * p.model.dof], np.float32), X[1])
    srv.close()


def test_shifted_tick_equals_host_shift(S):
    p = _mix(3)[2]
    srv = S.Server(MODELS, 2, 128, sqp_iters=3)
    sid = srv.open(p)
    r0 = srv.tick(sid, p.x_s, shift=False)
    X, U, lam = srv.read(sid)
    rng = np.random.default_rng(7)
    xs = X[1] + I.state_disturbance(rng, p.model.dof).astype(np.float32)
    srv.tick(sid, xs, shift=True)
    X1, U1, L1 = srv.read(sid)
    # the same tick on the host side: shift by one knot (last knot kept), new x_s
    Xs = np.concatenate([X[1:], X[-1:]])
    Us = np.concatenate([U[1:], U[-1:]])
    Ls = np.concatenate([lam[1:], lam[-1:]])
    q = I.Problem(p.model, p.N, p.dt, xs.astype(np.float64), p.cost_kind, p.w, x_ref=p.x_ref, seed=p.seed)
    g = gpu_solve(S.gato, [q], 3, X=[Xs], U=[Us], lam=[Ls])[0]
    np.testing.assert_array_equal(X1, g["X"].astype(np.float32))
    np.testing.assert_array_equal(U1, g["U"].astype(np.float32))
    assert r0.result.sqp_iters >= 1
    srv.close()


def test_same_result_alone_and_in_the_mix(S):
    probs = _mix(12)
    rng = np.random.default_rng(3)
    states = [p.x_s.astype(np.float32) + I.state_disturbance(rng, p.model.dof).astype(np.float32) for p in probs]
    # alone: one server, each session ticked by itself
    alone = []
    srv = S.Server(MODELS, 16, 128, sqp_iters=3, max_inflight=2)
    for p, x in zip(probs, states):
        sid = srv.open(p)
        srv.tick(sid, x, shift=True)
        alone.append(srv.read(sid))
    srv.close()
    # mixed: every session submitted at once, in two waves that overlap on the GPU
    srv = S.Server(MODELS, 16, 128, sqp_iters=3, max_inflight=2)
    sids = [srv.open(p) for p in probs]
    tickets = [srv.submit(s, x, True) for s, x in zip(sids[:6], states[:6])]
    tickets += [srv.submit(s, x, True) for s, x in zip(sids[6:], states[6:])]
    assert all(t is not None for t in tickets)
    for t in tickets:
        assert srv.poll(t, -1) is not None
    for i, s in enumerate(sids):
        X, U, L = srv.read(s)
        np.testing.assert_array_equal(X, alone[i][0])
        np.testing.assert_array_equal(U, alone[i][1])
        np.testing.assert_array_equal(L, alone[i][2])
    st = srv.stats()
    assert st["completed"] == 12 and st["launches"] >= 2
    srv.close()


def test_busy_session_and_admission_by_memory(S):
    probs = _mix(4)
    # a budget that holds the launch contexts and only a few slots
    srv = S.Server(MODELS, 1000, 128, max_batch=4, max_inflight=1, sqp_iters=1,
                   mem_budget_bytes=4 << 20)
    cap = srv.stats()["capacity"]
    assert 1 <= cap < 1000
    sids = []
    for i in range(cap):
        sids.append(srv.open(probs[i % 4]))
    assert all(s is not None for s in sids)
    assert srv.open(probs[0]) is None  # every slot taken
    srv.close_session(sids[0])
    assert srv.open(probs[0]) is not None
    t = srv.submit(sids[1], probs[1].x_s)
    assert t is not None
    assert srv.submit(sids[1], probs[1].x_s) is None  # ticks of a session are sequential
    assert srv.poll(t, -1) is not None
    srv.close()


def test_poisson_load_completes(S):
    probs = _mix(32)
    srv = S.Server(MODELS, 32, 128, sqp_iters=3, max_inflight=4)
    sids = [srv.open(p) for p in probs]
    out, lat = S.poisson_load(srv, sids, probs, rate=2000.0, duration_s=0.3, seed=5)
    assert out["completed"] == out["requests"] > 0
    assert (lat > 0).all() and out["p99_ms"] >= out["p50_ms"]
    srv.close()
