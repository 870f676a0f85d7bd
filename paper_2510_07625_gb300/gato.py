"""ctypes binding of ``include/gato.h`` (libgato.so).

The functions ``gato_*`` below carry the C names and only marshal arguments;
every step of the solver runs in the library's CUDA kernels.  ``Batch`` and
``DeviceProblems`` are conveniences that keep device buffers in torch tensors
(torch is used for memory and streams only).

Loading fails loudly when libgato.so is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as _inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgato.so")

GATO_OK, GATO_E_INVALID, GATO_E_NOMEM, GATO_E_CUDA, GATO_E_TIMEOUT, GATO_E_BUSY = 0, -1, -2, -3, -4, -5
SOLVE_CONVERGED, SOLVE_MAXITER, SOLVE_LSFAIL, SOLVE_PCG_MAXIT, SOLVE_NONFINITE = 1, 2, 4, 8, 16
COST_JOINT, COST_EE = 0, 1
PRECOND_STAIR, PRECOND_JACOBI = 0, 1
LINSOLVE_PCG, LINSOLVE_DIRECT = 0, 1
PRECISION_FP32, PRECISION_ESCALATE, PRECISION_HIGH = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1

EXPORTED = (
    "gato_default_params", "gato_create_batch", "gato_solve", "gato_step", "gato_solve_plain",
    "gato_sync", "gato_get_results", "gato_destroy_batch", "gato_status_string", "gato_last_error",
    "gato_last_transfer_bytes", "gato_debug_plain_stage", "gato_debug_layout", "gato_solve_noalloc",
    "gato_debug_stage_cycles", "gato_set_launch_config", "gato_autotune", "gato_graph_create",
    "gato_graph_launch", "gato_graph_wait", "gato_graph_destroy", "gato_server_create",
    "gato_server_open", "gato_server_submit", "gato_server_poll", "gato_server_read",
    "gato_server_close", "gato_server_get_stats", "gato_server_last_error", "gato_server_destroy",
    "gato_server_drive", "gato_query_launch", "gato_plant_rk4", "gato_plant_ee",
    "gato_debug_iteration_log",
)
LAYOUT_NAMES = ("X", "U", "dX", "dU", "Fq", "Fv", "Minv", "qdd", "dTau", "Qinv", "Rinv", "q", "r",
                "c", "Jk", "Linv", "links", "D", "L", "P", "vec", "scal", "Dx", "Du", "nu")


class ModelDesc(C.Structure):
    _fields_ = [("dof", C.c_int32), ("axis", C.c_int32 * 7), ("link_len", C.c_float * 7),
                ("mass", C.c_float * 7), ("com", C.c_float * 21), ("inertia", C.c_float * 21),
                ("gravity", C.c_float)]


class SolverParams(C.Structure):
    _fields_ = [("mu", C.c_float), ("beta", C.c_float), ("n_alpha", C.c_int32),
                ("pcg_eps", C.c_float), ("pcg_max_iter", C.c_int32), ("precond", C.c_int32),
                ("kkt_tol", C.c_float), ("linsolve", C.c_int32), ("rho_adapt", C.c_int32),
                ("precision", C.c_int32)]


class BatchDesc(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("max_horizon", C.c_int32), ("n_models", C.c_int32),
                ("models", C.POINTER(ModelDesc)), ("params", SolverParams)]


class Problem(C.Structure):
    _fields_ = [("model", C.c_int32), ("N", C.c_int32), ("dt", C.c_float),
                ("cost_kind", C.c_int32), ("w", C.c_float * 6), ("f_ext", C.c_float * 3),
                ("mem", C.c_int32),
                ("x_s", C.c_void_p), ("x_ref", C.c_void_p), ("ee_ref", C.c_void_p),
                ("X", C.c_void_p), ("U", C.c_void_p), ("lam", C.c_void_p)]


class LaunchConfig(C.Structure):
    _fields_ = [("variant", C.c_int32), ("knots_per_cta", C.c_int32), ("cluster", C.c_int32)]


class LaunchInfo(C.Structure):
    _fields_ = [("ctas_per_solve", C.c_int32), ("variant", C.c_int32), ("smem_bytes", C.c_int32),
                ("max_resident_solves", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("flags", C.c_int32), ("sqp_iters", C.c_int32), ("pcg_iters", C.c_int32),
                ("kkt_residual", C.c_float), ("merit", C.c_float)]


class ServerDesc(C.Structure):
    _fields_ = [("max_sessions", C.c_int32), ("max_horizon", C.c_int32), ("max_batch", C.c_int32),
                ("max_inflight", C.c_int32), ("sqp_iters", C.c_int32), ("mem_budget_bytes", C.c_int64)]


class Reply(C.Structure):
    _fields_ = [("result", Result), ("u0", C.c_float * 7), ("x1", C.c_float * 14),
                ("submit_ns", C.c_int64), ("done_ns", C.c_int64)]


class DriveStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("elapsed_s", C.c_double), ("launches", C.c_int64),
                ("max_backlog", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("sessions_open", C.c_int32), ("max_batch", C.c_int32),
                ("max_inflight", C.c_int32), ("submitted", C.c_int64), ("completed", C.c_int64),
                ("launches", C.c_int64), ("pending", C.c_int64), ("reserved_bytes", C.c_int64)]


_lib = None


def load() -> C.CDLL:
    """Loads libgato.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2510_07625_gb300.build` (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    bp = C.c_void_p
    L.gato_default_params.argtypes = [C.POINTER(SolverParams)]
    L.gato_default_params.restype = None
    L.gato_create_batch.argtypes = [C.POINTER(BatchDesc), C.c_void_p, C.POINTER(C.c_void_p)]
    L.gato_create_batch.restype = C.c_int
    for name in ("gato_solve", "gato_solve_plain"):
        f = getattr(L, name)
        f.argtypes = [bp, C.POINTER(Problem), C.c_int32, C.c_int32, C.POINTER(Result)]
        f.restype = C.c_int
    L.gato_step.argtypes = [bp, C.POINTER(Problem), C.c_int32, C.POINTER(Result)]
    L.gato_step.restype = C.c_int
    L.gato_sync.argtypes = [bp, C.c_int64]
    L.gato_sync.restype = C.c_int
    L.gato_get_results.argtypes = [bp, C.POINTER(Result), C.c_int32]
    L.gato_get_results.restype = C.c_int
    L.gato_destroy_batch.argtypes = [bp]
    L.gato_destroy_batch.restype = None
    L.gato_status_string.argtypes = [C.c_int]
    L.gato_status_string.restype = C.c_char_p
    L.gato_last_error.argtypes = [bp]
    L.gato_last_error.restype = C.c_char_p
    L.gato_last_transfer_bytes.argtypes = [bp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.gato_last_transfer_bytes.restype = C.c_int
    L.gato_debug_plain_stage.argtypes = [bp, C.POINTER(Problem), C.c_int32, C.c_void_p, C.c_int64]
    L.gato_debug_plain_stage.restype = C.c_int
    L.gato_debug_layout.argtypes = [bp, C.POINTER(C.c_int64)]
    L.gato_debug_layout.restype = C.c_int64
    L.gato_solve_noalloc.argtypes = [C.POINTER(ModelDesc), C.c_int32, C.POINTER(SolverParams),
                                     C.POINTER(Problem), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
    L.gato_solve_noalloc.restype = C.c_int
    L.gato_debug_stage_cycles.argtypes = [bp, C.c_int32, C.c_void_p, C.c_int32]
    L.gato_debug_stage_cycles.restype = C.c_int
    L.gato_debug_iteration_log.argtypes = [bp, C.c_int32, C.c_int32, C.c_void_p, C.c_int32]
    L.gato_debug_iteration_log.restype = C.c_int
    L.gato_set_launch_config.argtypes = [bp, C.POINTER(LaunchConfig)]
    L.gato_set_launch_config.restype = C.c_int
    L.gato_query_launch.argtypes = [C.c_int32, C.c_int32, C.POINTER(LaunchConfig), C.POINTER(LaunchInfo)]
    L.gato_query_launch.restype = C.c_int
    L.gato_autotune.argtypes = [bp, C.POINTER(Problem), C.c_int32, C.c_int32, C.c_int32,
                                C.POINTER(LaunchConfig), C.POINTER(C.c_float)]
    L.gato_autotune.restype = C.c_int
    L.gato_graph_create.argtypes = [bp, C.POINTER(Problem), C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]
    L.gato_graph_create.restype = C.c_int
    L.gato_graph_launch.argtypes = [bp, C.POINTER(Result)]
    L.gato_graph_launch.restype = C.c_int
    L.gato_graph_wait.argtypes = [bp, C.POINTER(Result)]
    L.gato_graph_wait.restype = C.c_int
    L.gato_graph_destroy.argtypes = [bp]
    L.gato_graph_destroy.restype = None
    L.gato_server_create.argtypes = [C.POINTER(BatchDesc), C.POINTER(ServerDesc), C.POINTER(C.c_void_p)]
    L.gato_server_create.restype = C.c_int
    L.gato_server_open.argtypes = [bp, C.POINTER(Problem), C.POINTER(C.c_int32)]
    L.gato_server_open.restype = C.c_int
    L.gato_server_submit.argtypes = [bp, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]
    L.gato_server_submit.restype = C.c_int
    L.gato_server_poll.argtypes = [bp, C.c_int64, C.c_int64, C.POINTER(Reply)]
    L.gato_server_poll.restype = C.c_int
    L.gato_server_read.argtypes = [bp, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.gato_server_read.restype = C.c_int
    L.gato_server_close.argtypes = [bp, C.c_int32]
    L.gato_server_close.restype = C.c_int
    L.gato_server_get_stats.argtypes = [bp, C.POINTER(ServerStats)]
    L.gato_server_get_stats.restype = C.c_int
    L.gato_server_last_error.argtypes = [bp]
    L.gato_server_last_error.restype = C.c_char_p
    L.gato_server_destroy.argtypes = [bp]
    L.gato_server_destroy.restype = None
    L.gato_server_drive.argtypes = [bp, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(DriveStats)]
    L.gato_server_drive.restype = C.c_int
    dp = C.POINTER(C.c_double)
    L.gato_plant_rk4.argtypes = [C.POINTER(ModelDesc), dp, dp, dp, C.c_double, C.c_int32, dp]
    L.gato_plant_rk4.restype = C.c_int
    L.gato_plant_ee.argtypes = [C.POINTER(ModelDesc), dp, dp]
    L.gato_plant_ee.restype = C.c_int
    _lib = L
    return L


class GatoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


# ----------------------------------------------------------- C-named wrappers

def gato_default_params() -> SolverParams:
    p = SolverParams()
    load().gato_default_params(C.byref(p))
    return p


def gato_status_string(s: int) -> str:
    return load().gato_status_string(s).decode()


def gato_create_batch(desc: BatchDesc, stream: int | None = None) -> int:
    h = C.c_void_p()
    s = load().gato_create_batch(C.byref(desc), C.c_void_p(stream or 0), C.byref(h))
    if s != GATO_OK:
        raise GatoError(s, f"gato_create_batch: {gato_status_string(s)}")
    return h.value


def _check(handle, s, what):
    if s != GATO_OK:
        msg = load().gato_last_error(C.c_void_p(handle)).decode()
        raise GatoError(s, f"{what}: {gato_status_string(s)}: {msg}")


def gato_solve(handle, problems, n, iters, results=None):
    r = results if results is not None else None
    s = load().gato_solve(C.c_void_p(handle), problems, n, iters, r)
    _check(handle, s, "gato_solve")


def gato_step(handle, problems, n, results=None):
    s = load().gato_step(C.c_void_p(handle), problems, n, results)
    _check(handle, s, "gato_step")


def gato_solve_plain(handle, problems, n, iters, results=None):
    s = load().gato_solve_plain(C.c_void_p(handle), problems, n, iters, results)
    _check(handle, s, "gato_solve_plain")


def gato_sync(handle, timeout_us=-1) -> int:
    s = load().gato_sync(C.c_void_p(handle), timeout_us)
    if s not in (GATO_OK, GATO_E_TIMEOUT):
        _check(handle, s, "gato_sync")
    return s


def gato_get_results(handle, n):
    out = (Result * n)()
    s = load().gato_get_results(C.c_void_p(handle), out, n)
    _check(handle, s, "gato_get_results")
    return out


def gato_destroy_batch(handle):
    load().gato_destroy_batch(C.c_void_p(handle))


def gato_last_error(handle) -> str:
    return load().gato_last_error(C.c_void_p(handle)).decode()


def gato_last_transfer_bytes(handle):
    a, b = C.c_int64(), C.c_int64()
    load().gato_last_transfer_bytes(C.c_void_p(handle), C.byref(a), C.byref(b))
    return a.value, b.value


def gato_debug_layout(handle):
    off = (C.c_int64 * 25)()
    total = load().gato_debug_layout(C.c_void_p(handle), off)
    return total, dict(zip(LAYOUT_NAMES, list(off)))


def gato_debug_plain_stage(handle, problems, stop_stage):
    total, off = gato_debug_layout(handle)
    buf = np.zeros(total, np.float32)
    s = load().gato_debug_plain_stage(C.c_void_p(handle), problems, stop_stage,
                                      buf.ctypes.data_as(C.c_void_p), total)
    _check(handle, s, "gato_debug_plain_stage")
    return buf, off


STAGE_NAMES = ("load", "mass", "fd", "value_cost", "tangents", "jacobians", "kkt", "schur",
               "block_inverse", "pcg_init", "pcg_S", "pcg_y", "pcg_wz", "recover", "line_search",
               "accept")


def gato_debug_stage_cycles(handle, enable, n=0):
    """enable=1: start counting; enable=0: return an (n, 16) array of cycles and stop."""
    out = np.zeros((max(n, 1), 16), np.int64)
    s = load().gato_debug_stage_cycles(C.c_void_p(handle), enable,
                                       out.ctypes.data if (not enable and n) else None, n)
    _check(handle, s, "gato_debug_stage_cycles")
    return None if enable else out[:n]


def gato_debug_iteration_log(handle, enable, max_iters, n=0):
    """enable=1: start logging max_iters iterations per solve; enable=0: return
    a dict of (n, max_iters) arrays (alpha index, PCG iterations, KKT residual,
    high-precision flag, merit of the iterate, merit of the full step) and stop."""
    out = np.zeros((max(n, 1), max_iters, 8), np.int32)
    s = load().gato_debug_iteration_log(C.c_void_p(handle), enable, max_iters,
                                        out.ctypes.data if (not enable and n) else None, n)
    _check(handle, s, "gato_debug_iteration_log")
    if enable:
        return None
    out = out[:n]
    f = out.view(np.float32).astype(np.float64)
    return {"alpha_idx": out[:, :, 0].copy(), "pcg_iters": out[:, :, 1].copy(),
            "kkt": out[:, :, 2].copy().view(np.float32), "hp": out[:, :, 3].copy(),
            "merit": f[:, :, 4] + f[:, :, 5], "merit_full_step": f[:, :, 6] + f[:, :, 7]}


def gato_solve_noalloc(models, n_models, params, problems, n, iters, results_dev_ptr, stream=0):
    """Allocation-free solve: device problems only, results written to device memory."""
    s = load().gato_solve_noalloc(models, n_models, C.byref(params), problems, n, iters,
                                  C.c_void_p(results_dev_ptr), C.c_void_p(stream or 0))
    if s != GATO_OK:
        raise GatoError(s, f"gato_solve_noalloc: {gato_status_string(s)}")


def gato_query_launch(N, n_solves, variant=None, knots_per_cta=0, cluster=0):
    """Launch shape of n_solves solves of horizon N on the current device
    (variant None = the automatic configuration): a dict with ctas_per_solve,
    variant, smem_bytes and max_resident_solves."""
    info = LaunchInfo()
    cfg = None if variant is None else C.byref(LaunchConfig(variant, knots_per_cta, cluster))
    s = load().gato_query_launch(N, n_solves, cfg, C.byref(info))
    if s != GATO_OK:
        raise GatoError(s, f"gato_query_launch: {gato_status_string(s)}")
    return {f: getattr(info, f) for f, _ in LaunchInfo._fields_}


def gato_set_launch_config(handle, variant=None, knots_per_cta=0, cluster=0):
    """variant None clears the forced configuration."""
    if variant is None:
        s = load().gato_set_launch_config(C.c_void_p(handle), None)
    else:
        cfg = LaunchConfig(variant, knots_per_cta, cluster)
        s = load().gato_set_launch_config(C.c_void_p(handle), C.byref(cfg))
    _check(handle, s, "gato_set_launch_config")


def gato_autotune(handle, problems, n, iters, reps=3):
    cfg, ms = LaunchConfig(), C.c_float()
    s = load().gato_autotune(C.c_void_p(handle), problems, n, iters, reps, C.byref(cfg), C.byref(ms))
    _check(handle, s, "gato_autotune")
    return dict(variant=cfg.variant, knots_per_cta=cfg.knots_per_cta, cluster=cfg.cluster), ms.value


def gato_graph_create(handle, problems, n, iters) -> int:
    g = C.c_void_p()
    s = load().gato_graph_create(C.c_void_p(handle), problems, n, iters, C.byref(g))
    _check(handle, s, "gato_graph_create")
    return g.value


def gato_graph_launch(graph, results=None):
    s = load().gato_graph_launch(C.c_void_p(graph), results)
    if s != GATO_OK:
        raise GatoError(s, f"gato_graph_launch: {gato_status_string(s)}")


def gato_graph_wait(graph, results=None):
    s = load().gato_graph_wait(C.c_void_p(graph), results)
    if s != GATO_OK:
        raise GatoError(s, f"gato_graph_wait: {gato_status_string(s)}")


def gato_graph_destroy(graph):
    load().gato_graph_destroy(C.c_void_p(graph))


def _scheck(handle, s, what, ok=(GATO_OK,)):
    if s not in ok:
        msg = load().gato_server_last_error(C.c_void_p(handle)).decode()
        raise GatoError(s, f"{what}: {gato_status_string(s)}: {msg}")
    return s


def gato_server_create(desc: BatchDesc, sdesc: ServerDesc) -> int:
    h = C.c_void_p()
    s = load().gato_server_create(C.byref(desc), C.byref(sdesc), C.byref(h))
    if s != GATO_OK:
        raise GatoError(s, f"gato_server_create: {gato_status_string(s)}")
    return h.value


def gato_server_open(handle, problem) -> int | None:
    """Session id, or None when every slot is taken (GATO_E_BUSY)."""
    sid = C.c_int32()
    s = load().gato_server_open(C.c_void_p(handle), C.byref(problem), C.byref(sid))
    if _scheck(handle, s, "gato_server_open", (GATO_OK, GATO_E_BUSY)) == GATO_E_BUSY:
        return None
    return sid.value


def gato_server_submit(handle, session, x_s, shift=True) -> int | None:
    """Ticket, or None when the session still has a request (GATO_E_BUSY)."""
    xs = np.ascontiguousarray(x_s, np.float32)
    t = C.c_int64()
    s = load().gato_server_submit(C.c_void_p(handle), session, xs.ctypes.data, 1 if shift else 0, C.byref(t))
    if _scheck(handle, s, "gato_server_submit", (GATO_OK, GATO_E_BUSY)) == GATO_E_BUSY:
        return None
    return t.value


def gato_server_poll(handle, ticket, timeout_us=-1):
    """The Reply, or None if not done within the timeout."""
    r = Reply()
    s = load().gato_server_poll(C.c_void_p(handle), ticket, timeout_us, C.byref(r))
    if _scheck(handle, s, "gato_server_poll", (GATO_OK, GATO_E_TIMEOUT)) == GATO_E_TIMEOUT:
        return None
    return r


def gato_server_read(handle, session, N, dof):
    X = np.zeros((N + 1, 2 * dof), np.float32)
    U = np.zeros((N, dof), np.float32)
    lam = np.zeros((N + 1, 2 * dof), np.float32)
    s = load().gato_server_read(C.c_void_p(handle), session, X.ctypes.data, U.ctypes.data, lam.ctypes.data)
    _scheck(handle, s, "gato_server_read")
    return X, U, lam


def gato_server_close(handle, session):
    _scheck(handle, load().gato_server_close(C.c_void_p(handle), session), "gato_server_close")


def gato_server_get_stats(handle) -> dict:
    st = ServerStats()
    _scheck(handle, load().gato_server_get_stats(C.c_void_p(handle), C.byref(st)), "gato_server_get_stats")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def gato_server_destroy(handle):
    load().gato_server_destroy(C.c_void_p(handle))


def gato_server_drive(handle, sessions, x_init, t_arrival, client, noise):
    """Replays an arrival schedule; returns (latency_ms array, stats dict)."""
    sess = np.ascontiguousarray(sessions, np.int32)
    x0 = np.ascontiguousarray(x_init, np.float32).reshape(len(sess), 14)
    t = np.ascontiguousarray(t_arrival, np.float64)
    cl = np.ascontiguousarray(client, np.int32)
    nz = np.ascontiguousarray(noise, np.float32).reshape(len(t), 14)
    lat = np.zeros(len(t), np.float32)
    st = DriveStats()
    s = load().gato_server_drive(C.c_void_p(handle), sess.ctypes.data, len(sess), x0.ctypes.data,
                                 t.ctypes.data, cl.ctypes.data, nz.ctypes.data, len(t), lat.ctypes.data,
                                 C.byref(st))
    _scheck(handle, s, "gato_server_drive")
    return lat, {k: getattr(st, k) for k, _ in DriveStats._fields_}


# ------------------------------------------------------------- conveniences

def model_desc(m) -> ModelDesc:
    d = ModelDesc()
    d.dof = m.dof
    for i in range(7):
        d.axis[i] = m.axis[i] if i < m.dof else 2
        d.link_len[i] = m.link_len[i] if i < m.dof else 0.0
        d.mass[i] = m.mass[i] if i < m.dof else 0.0
    for i in range(21):
        d.com[i] = m.com[i] if i < 3 * m.dof else 0.0
        d.inertia[i] = m.inertia[i] if i < 3 * m.dof else 0.0
    d.gravity = m.gravity
    return d


def results_to_dicts(res, n):
    return [dict(flags=res[i].flags, sqp_iters=res[i].sqp_iters, pcg_iters=res[i].pcg_iters,
                 kkt=res[i].kkt_residual, merit=res[i].merit) for i in range(n)]


class Batch:
    """Owns a gato_batch handle for a fixed set of models."""

    def __init__(self, models, max_batch, max_horizon, params: SolverParams | None = None,
                 stream: int | None = None, **overrides):
        self.models = list(models)
        self._mdesc = (ModelDesc * len(self.models))(*[model_desc(m) for m in self.models])
        p = params or gato_default_params()
        for k, v in overrides.items():
            setattr(p, k, v)
        self.params = p
        d = BatchDesc(max_batch, max_horizon, len(self.models),
                      C.cast(self._mdesc, C.POINTER(ModelDesc)), p)
        self.handle = gato_create_batch(d, stream)
        self.max_batch = max_batch
        self.max_horizon = max_horizon

    def model_index(self, m):
        for i, mm in enumerate(self.models):
            if mm == m:
                return i
        raise KeyError(f"model {m.name} not in batch")

    def solve(self, problems, n, iters, plain=False):
        res = (Result * n)()
        f = gato_solve_plain if plain else gato_solve
        f(self.handle, problems, n, iters, res)
        return res

    def solve_async(self, problems, n, iters):
        gato_solve(self.handle, problems, n, iters, None)

    def set_launch_config(self, variant=None, knots_per_cta=0, cluster=0):
        gato_set_launch_config(self.handle, variant, knots_per_cta, cluster)

    def autotune(self, problems, n, iters, reps=3):
        """Times the launch configurations on these problems; returns (config, median ms)."""
        return gato_autotune(self.handle, problems, n, iters, reps)

    def capture(self, problems, n, iters):
        """A CUDA graph of one solve call on device problems."""
        return Graph(self, problems, n, iters)

    def sync(self, timeout_us=-1):
        return gato_sync(self.handle, timeout_us)

    def close(self):
        if getattr(self, "handle", None):
            gato_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured solve (gato_graph_*); replay() returns the per-solve results."""

    def __init__(self, batch: Batch, problems, n, iters):
        self.batch = batch
        self.n = n
        self.handle = gato_graph_create(batch.handle, problems, n, iters)

    def replay(self, wait=True):
        if not wait:
            gato_graph_launch(self.handle, None)
            return None
        res = (Result * self.n)()
        gato_graph_launch(self.handle, res)
        return res

    def wait(self):
        res = (Result * self.n)()
        gato_graph_wait(self.handle, res)
        return res

    def close(self):
        if getattr(self, "handle", None):
            gato_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cold_start_arrays(prob):
    """Cold-start initial guess (the paper gives none): X_k = x_s, U = 0, lambda = 0 (float32)."""
    nx, nu = 2 * prob.model.dof, prob.model.dof
    X = np.tile(np.asarray(prob.x_s, np.float32), (prob.N + 1, 1))
    U = np.zeros((prob.N, nu), np.float32)
    lam = np.zeros((prob.N + 1, nx), np.float32)
    return X, U, lam


class HostProblems:
    """gato_problem array over numpy (host) buffers; X/U/lambda updated in place."""

    def __init__(self, batch: Batch, probs, X=None, U=None, lam=None):
        self.probs = list(probs)
        n = len(self.probs)
        self.arr = (Problem * n)()
        self.keep = []
        self.X, self.U, self.lam = [], [], []
        for i, p in enumerate(self.probs):
            X0, U0, L0 = cold_start_arrays(p)
            Xi = np.ascontiguousarray(X[i] if X is not None else X0, np.float32)
            Ui = np.ascontiguousarray(U[i] if U is not None else U0, np.float32)
            Li = np.ascontiguousarray(lam[i] if lam is not None else L0, np.float32)
            xs = np.ascontiguousarray(p.x_s, np.float32)
            ref = np.ascontiguousarray(p.x_ref if p.cost_kind == COST_JOINT else p.ee_ref, np.float32)
            self.keep += [xs, ref]
            self.X.append(Xi)
            self.U.append(Ui)
            self.lam.append(Li)
            a = self.arr[i]
            a.model = batch.model_index(p.model)
            a.N = p.N
            a.dt = p.dt
            a.cost_kind = p.cost_kind
            for k in range(6):
                a.w[k] = p.w[k]
            for k, f in enumerate(getattr(p, "f_ext", (0.0, 0.0, 0.0))):
                a.f_ext[k] = f
            a.mem = MEM_HOST
            a.x_s = xs.ctypes.data
            a.x_ref = ref.ctypes.data if p.cost_kind == COST_JOINT else None
            a.ee_ref = ref.ctypes.data if p.cost_kind == COST_EE else None
            a.X = Xi.ctypes.data
            a.U = Ui.ctypes.data
            a.lam = Li.ctypes.data
        self.n = n


class DeviceProblems:
    """gato_problem array over torch CUDA tensors (padded [B, Nmax+1, nx] slabs)."""

    def __init__(self, batch: Batch, probs, device="cuda"):
        import torch

        self.torch = torch
        self.probs = list(probs)
        n = len(self.probs)
        Nmax = max(p.N for p in self.probs)
        self.Nmax = Nmax
        f32 = torch.float32
        self.x_s = torch.zeros(n, 14, dtype=f32, device=device)
        self.ref = torch.zeros(n, (Nmax + 1) * 14, dtype=f32, device=device)
        self.X = torch.zeros(n, (Nmax + 1) * 14, dtype=f32, device=device)
        self.U = torch.zeros(n, Nmax * 7, dtype=f32, device=device)
        self.lam = torch.zeros(n, (Nmax + 1) * 14, dtype=f32, device=device)
        self.arr = (Problem * n)()
        hx = np.zeros((n, 14), np.float32)
        href = np.zeros((n, (Nmax + 1) * 14), np.float32)
        hX = np.zeros((n, (Nmax + 1) * 14), np.float32)
        for i, p in enumerate(self.probs):
            nx = 2 * p.model.dof
            hx[i, :nx] = p.x_s
            r = p.x_ref if p.cost_kind == COST_JOINT else p.ee_ref
            r = np.asarray(r, np.float32).ravel()
            href[i, :r.size] = r
            X0, _, _ = cold_start_arrays(p)
            hX[i, :X0.size] = X0.ravel()
        self.x_s.copy_(torch.from_numpy(hx))
        self.ref.copy_(torch.from_numpy(href))
        self.X.copy_(torch.from_numpy(hX))
        es = 4
        for i, p in enumerate(self.probs):
            a = self.arr[i]
            a.model = batch.model_index(p.model)
            a.N = p.N
            a.dt = p.dt
            a.cost_kind = p.cost_kind
            for k in range(6):
                a.w[k] = p.w[k]
            for k, f in enumerate(getattr(p, "f_ext", (0.0, 0.0, 0.0))):
                a.f_ext[k] = f
            a.mem = MEM_DEVICE
            a.x_s = self.x_s.data_ptr() + i * 14 * es
            rp = self.ref.data_ptr() + i * (Nmax + 1) * 14 * es
            a.x_ref = rp if p.cost_kind == COST_JOINT else None
            a.ee_ref = rp if p.cost_kind == COST_EE else None
            a.X = self.X.data_ptr() + i * (Nmax + 1) * 14 * es
            a.U = self.U.data_ptr() + i * Nmax * 7 * es
            a.lam = self.lam.data_ptr() + i * (Nmax + 1) * 14 * es
        self.n = n
        self._X0 = self.X.clone()

    def reset(self):
        """Back to the cold start (X = x_s, U = 0, lambda = 0)."""
        self.X.copy_(self._X0)
        self.U.zero_()
        self.lam.zero_()

    def solution(self, i):
        p = self.probs[i]
        nx, nu = 2 * p.model.dof, p.model.dof
        X = self.X[i, : (p.N + 1) * nx].reshape(p.N + 1, nx).double().cpu().numpy()
        U = self.U[i, : p.N * nu].reshape(p.N, nu).double().cpu().numpy()
        L = self.lam[i, : (p.N + 1) * nx].reshape(p.N + 1, nx).double().cpu().numpy()
        return X, U, L


# ------------------------------------------------------------------ plant

def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Plant:
    """The simulated robot of closed-loop runs (host, double): RK4 of the
    rigid-body dynamics with an end-effector force (gato_plant_rk4)."""

    def __init__(self, model):
        self.model = model
        self.desc = model_desc(model)
        self.lib = load()

    def rk4(self, x, u, h, steps, f_ext=None):
        x = np.ascontiguousarray(x, np.float64)
        u = np.ascontiguousarray(u, np.float64)
        out = np.empty_like(x)
        fe = None if f_ext is None else np.ascontiguousarray(f_ext, np.float64)
        st = self.lib.gato_plant_rk4(C.byref(self.desc), _dptr(x), _dptr(u),
                                     _dptr(fe) if fe is not None else None, h, steps, _dptr(out))
        if st != 0:
            raise GatoError(st, "gato_plant_rk4 failed")
        return out

    def ee(self, q):
        q = np.ascontiguousarray(q, np.float64)
        p = np.empty(3)
        st = self.lib.gato_plant_ee(C.byref(self.desc), _dptr(q), _dptr(p))
        if st != 0:
            raise GatoError(st, "gato_plant_ee failed")
        return p
