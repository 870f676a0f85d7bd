"""Serving loop over the C ABI: continuous batching of MPC control ticks.

``Server`` wraps ``gato_server_*``: sessions (one resident warm-started
trajectory each) are admitted while the device-memory budget has slots; each
request is one control tick (new measured state, one-knot warm-start shift,
a fixed number of SQP iterations).  The library's worker thread launches all
pending requests together whenever a launch context is free, so requests
that arrive while others run join the next launch and overlap on the GPU.

``poisson_load`` replays Poisson arrivals of ticks over the sessions through
the library's load driver and reports solves/s and latency percentiles.
"""
from __future__ import annotations

import numpy as np

from . import gato, inputs as I


class Server:
    def __init__(self, models, max_sessions, max_horizon, max_batch=256, max_inflight=4, sqp_iters=3,
                 mem_budget_bytes=0, params=None, **overrides):
        self.models = list(models)
        self._mdesc = (gato.ModelDesc * len(self.models))(*[gato.model_desc(m) for m in self.models])
        p = params or gato.gato_default_params()
        for k, v in overrides.items():
            setattr(p, k, v)
        import ctypes as C

        d = gato.BatchDesc(1, max_horizon, len(self.models), C.cast(self._mdesc, C.POINTER(gato.ModelDesc)), p)
        sd = gato.ServerDesc(max_sessions, max_horizon, max_batch, max_inflight, sqp_iters, mem_budget_bytes)
        self.handle = gato.gato_server_create(d, sd)
        self.sqp_iters = sqp_iters
        self._sessions = {}

    def open(self, prob, X=None, U=None, lam=None):
        """Session id for a problem (host data copied in), or None if no slot is free."""
        hp = _HostProblem(self, prob, X, U, lam)
        sid = gato.gato_server_open(self.handle, hp.arr)
        if sid is not None:
            self._sessions[sid] = prob
        return sid

    def submit(self, sid, x_s, shift=True):
        return gato.gato_server_submit(self.handle, sid, x_s, shift)

    def poll(self, ticket, timeout_us=-1):
        return gato.gato_server_poll(self.handle, ticket, timeout_us)

    def tick(self, sid, x_s, shift=True):
        """One synchronous control tick; returns the Reply."""
        t = self.submit(sid, x_s, shift)
        if t is None:
            raise gato.GatoError(gato.GATO_E_BUSY, "session busy")
        return self.poll(t, -1)

    def read(self, sid):
        p = self._sessions[sid]
        return gato.gato_server_read(self.handle, sid, p.N, p.model.dof)

    def close_session(self, sid):
        gato.gato_server_close(self.handle, sid)
        self._sessions.pop(sid, None)

    def stats(self):
        return gato.gato_server_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            gato.gato_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _HostProblem:
    def __init__(self, server, prob, X, U, lam):
        import ctypes as C

        self.keep = []
        a = gato.Problem()
        a.model = server.models.index(prob.model)
        a.N = prob.N
        a.dt = prob.dt
        a.cost_kind = prob.cost_kind
        for k in range(6):
            a.w[k] = prob.w[k]
        for k, f in enumerate(getattr(prob, "f_ext", (0.0, 0.0, 0.0))):
            a.f_ext[k] = f
        a.mem = gato.MEM_HOST
        xs = np.ascontiguousarray(prob.x_s, np.float32)
        ref = np.ascontiguousarray(prob.x_ref if prob.cost_kind == gato.COST_JOINT else prob.ee_ref, np.float32)
        self.keep += [xs, ref]
        a.x_s = xs.ctypes.data
        a.x_ref = ref.ctypes.data if prob.cost_kind == gato.COST_JOINT else None
        a.ee_ref = ref.ctypes.data if prob.cost_kind == gato.COST_EE else None
        for name, v in (("X", X), ("U", U), ("lam", lam)):
            if v is None:
                setattr(a, name, None)
            else:
                arr = np.ascontiguousarray(v, np.float32)
                self.keep.append(arr)
                setattr(a, name, arr.ctypes.data)
        self.arr = a


def poisson_load(server: Server, sids, probs, rate, duration_s, seed=12345, sigma_q=0.05, sigma_qd=0.1,
                 max_requests=None):
    """Poisson ticks at `rate` requests/s over the open sessions `sids`, for
    `duration_s` seconds or `max_requests` arrivals, whichever comes first.

    Each arrival is a tick of a uniformly drawn session: its last predicted
    state plus Gaussian disturbance (sigma_q rad, sigma_qd rad/s), warm start
    shifted one knot.  Latency runs from the scheduled arrival to completion.
    """
    t, clients = I.poisson_arrivals(rate, duration_s, len(sids), seed=seed, max_requests=max_requests)
    rng = np.random.default_rng(seed + 1)
    noise = np.zeros((len(t), 14), np.float32)
    for i, c in enumerate(clients):
        nq = probs[c].model.dof
        d = I.state_disturbance(rng, nq, sigma_q, sigma_qd)
        noise[i, :2 * nq] = d
    x0 = np.zeros((len(sids), 14), np.float32)
    for c, p in enumerate(probs):
        x0[c, :2 * p.model.dof] = p.x_s
    lat, st = gato.gato_server_drive(server.handle, sids, x0, t, clients, noise)
    done = lat[:st["completed"]] if st["completed"] == len(t) else lat
    out = {"rate_req_s": rate, "requests": int(len(t)), "completed": int(st["completed"]),
           "elapsed_s": round(st["elapsed_s"], 4),
           "solves_per_s": round(st["completed"] / st["elapsed_s"], 1) if st["elapsed_s"] > 0 else 0.0,
           "p50_ms": round(float(np.percentile(done, 50)), 4) if len(done) else None,
           "p99_ms": round(float(np.percentile(done, 99)), 4) if len(done) else None,
           "launches": int(st["launches"]),
           "mean_batch": round(st["completed"] / max(1, st["launches"]), 2),
           "max_backlog": int(st["max_backlog"])}
    return out, lat
