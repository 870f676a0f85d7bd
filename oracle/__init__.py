"""FP64 CPU oracle for the batched SQP method (GATO, arXiv 2510.07625).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA product path
never imports this package, and this package never imports the product.

The arithmetic lives in ``gato_oracle.cpp`` (plain C++17, double precision);
this module compiles it with the host compiler and wraps it with ctypes.
Every function takes numpy arrays in the problem's own sizes
(nx = 2 * dof, nu = dof, no padding).

Parity of the full nonlinear SQP path (line search on the nonlinear arm) is
pinned only by invariants and by the dense/LQR special cases; the dynamics,
Schur blocks, preconditioner, PCG and recovery are pinned directly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gato_oracle.cpp")
_LIB = os.path.join(_HERE, "libgato_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_CONVERGED, FLAG_MAXITER, FLAG_LSFAIL, FLAG_PCG_MAXIT, FLAG_NONFINITE = 1, 2, 4, 8, 16


class OraModel(C.Structure):
    _fields_ = [("dof", C.c_int32), ("axis", C.c_int32 * 7), ("link_len", C.c_double * 7),
                ("mass", C.c_double * 7), ("com", C.c_double * 21),
                ("inertia", C.c_double * 21), ("gravity", C.c_double)]


class OraProblem(C.Structure):
    _fields_ = [("N", C.c_int32), ("cost_kind", C.c_int32), ("dt", C.c_double),
                ("x_s", C.POINTER(C.c_double)), ("x_ref", C.POINTER(C.c_double)),
                ("ee_ref", C.POINTER(C.c_double)), ("w", C.c_double * 6),
                ("f_ext", C.c_double * 3)]


class OraParams(C.Structure):
    _fields_ = [("mu", C.c_double), ("beta", C.c_double), ("n_alpha", C.c_int32),
                ("pcg_eps", C.c_double), ("pcg_max", C.c_int32), ("precond", C.c_int32),
                ("kkt_tol", C.c_double), ("max_iter", C.c_int32), ("linsolve", C.c_int32),
                ("rho_adapt", C.c_int32)]


class OraResult(C.Structure):
    _fields_ = [("iters", C.c_int32), ("flags", C.c_int32), ("pcg_total", C.c_int32),
                ("kkt", C.c_double), ("merit", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``libgato_oracle.so`` beside its source."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        mp = C.POINTER(OraModel)
        pp = C.POINTER(OraProblem)
        L.ora_rnea.argtypes = [mp, dp, dp, dp, C.c_int32, dp]
        L.ora_mass_matrix.argtypes = [mp, dp, dp]
        L.ora_forward_dynamics.argtypes = [mp, dp, dp, dp, dp, dp]
        L.ora_forward_dynamics.restype = C.c_int32
        L.ora_step.argtypes = [mp, dp, dp, C.c_double, dp, dp]
        L.ora_step.restype = C.c_int32
        L.ora_step_jacobians.argtypes = [mp, dp, dp, C.c_double, dp, dp, dp]
        L.ora_ee_joint_torque.argtypes = [mp, dp, dp, dp]
        L.ora_fk.argtypes = [mp, dp, dp, dp]
        L.ora_merit.argtypes = [mp, pp, dp, dp, C.c_double]
        L.ora_merit.restype = C.c_double
        L.ora_linearize.argtypes = [mp, pp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.ora_linearize.restype = C.c_double
        L.ora_schur.argtypes = [mp, pp, dp, dp, C.c_int32, dp, dp, dp, dp, dp]
        L.ora_schur.restype = C.c_int32
        L.ora_pcg.argtypes = [C.c_int32, C.c_int32, dp, dp, dp, dp, dp, C.c_double, C.c_int32, dp]
        L.ora_pcg.restype = C.c_int32
        L.ora_qp_step.argtypes = [mp, pp, dp, dp, C.c_int32, C.c_double, C.c_int32, dp, dp, dp]
        L.ora_qp_step.restype = C.c_int32
        L.ora_kkt_residual.argtypes = [mp, pp, dp, dp, dp]
        L.ora_kkt_residual.restype = C.c_double
        L.ora_solve.argtypes = [mp, pp, C.POINTER(OraParams), dp, dp, dp, ip, ip, ip, dp, dp, dp,
                                dp, C.POINTER(OraResult)]
        L.ora_solve.restype = C.c_int32
        L.ora_blocktri_solve.argtypes = [C.c_int32, C.c_int32, dp, dp, dp, dp]
        L.ora_blocktri_solve.restype = C.c_int32
        L.ora_count_flops.argtypes = [mp, C.c_int32]
        L.ora_count_flops.restype = C.c_int64
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _arr(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_model(model) -> OraModel:
    """Convert an ``inputs.ArmModel`` (or anything with the same fields)."""
    m = OraModel()
    m.dof = model.dof
    for i in range(7):
        m.axis[i] = model.axis[i] if i < model.dof else 2
        m.link_len[i] = model.link_len[i] if i < model.dof else 0.0
        m.mass[i] = model.mass[i] if i < model.dof else 0.0
    for i in range(21):
        m.com[i] = model.com[i] if i < 3 * model.dof else 0.0
        m.inertia[i] = model.inertia[i] if i < 3 * model.dof else 0.0
    m.gravity = model.gravity
    return m


class _Prob:
    """Keeps the numpy buffers of an OraProblem alive."""

    def __init__(self, prob):
        self.model = make_model(prob.model)
        self.x_s = _arr(prob.x_s)
        self.x_ref = None if prob.x_ref is None else _arr(prob.x_ref)
        self.ee_ref = None if prob.ee_ref is None else _arr(prob.ee_ref)
        p = OraProblem()
        p.N = prob.N
        p.cost_kind = prob.cost_kind
        p.dt = prob.dt
        p.x_s = _d(self.x_s)
        p.x_ref = _d(self.x_ref) if self.x_ref is not None else C.POINTER(C.c_double)()
        p.ee_ref = _d(self.ee_ref) if self.ee_ref is not None else C.POINTER(C.c_double)()
        for i in range(6):
            p.w[i] = prob.w[i]
        for i, f in enumerate(getattr(prob, "f_ext", (0.0, 0.0, 0.0))):
            p.f_ext[i] = f
        self.p = p
        self.N = prob.N
        self.nx = 2 * prob.model.dof
        self.nu = prob.model.dof


# ----------------------------------------------------------------- dynamics

def rnea(model, q, qd, qdd, gravity=True):
    n = model.dof
    q, qd, qdd = _arr(q), _arr(qd), _arr(qdd)
    tau = np.zeros(n)
    m = make_model(model)
    lib().ora_rnea(C.byref(m), _d(q), _d(qd), _d(qdd), 1 if gravity else 0, _d(tau))
    return tau


def mass_matrix(model, q):
    n = model.dof
    M = np.zeros((n, n))
    m = make_model(model)
    lib().ora_mass_matrix(C.byref(m), _d(_arr(q)), _d(M))
    return M


def _fext(f_ext):
    return C.POINTER(C.c_double)() if f_ext is None else _d(_arr(f_ext))


def forward_dynamics(model, q, qd, tau, f_ext=None):
    """qdd from M(q) qdd = tau + J_p(q)^T f_ext - ID(q, qd, 0)."""
    n = model.dof
    out = np.zeros(n)
    m = make_model(model)
    fe = None if f_ext is None else _arr(f_ext)
    rc = lib().ora_forward_dynamics(C.byref(m), _d(_arr(q)), _d(_arr(qd)), _d(_arr(tau)),
                                    _fext(fe), _d(out))
    if rc != 0:
        raise FloatingPointError("mass matrix not positive definite")
    return out


def step(model, x, u, h, f_ext=None):
    out = np.zeros(2 * model.dof)
    m = make_model(model)
    fe = None if f_ext is None else _arr(f_ext)
    lib().ora_step(C.byref(m), _d(_arr(x)), _d(_arr(u)), h, _fext(fe), _d(out))
    return out


def step_jacobians(model, x, u, h, f_ext=None):
    nx, nu = 2 * model.dof, model.dof
    A = np.zeros((nx, nx))
    B = np.zeros((nx, nu))
    m = make_model(model)
    fe = None if f_ext is None else _arr(f_ext)
    lib().ora_step_jacobians(C.byref(m), _d(_arr(x)), _d(_arr(u)), h, _fext(fe), _d(A), _d(B))
    return A, B


def ee_joint_torque(model, q, f):
    """J_p(q)^T f: joint torques of a base-frame force f at the end effector."""
    tau = np.zeros(model.dof)
    m = make_model(model)
    lib().ora_ee_joint_torque(C.byref(m), _d(_arr(q)), _d(_arr(f)), _d(tau))
    return tau


def fk(model, q, jacobian=False):
    p = np.zeros(3)
    m = make_model(model)
    if jacobian:
        J = np.zeros((3, model.dof))
        lib().ora_fk(C.byref(m), _d(_arr(q)), _d(p), _d(J))
        return p, J
    lib().ora_fk(C.byref(m), _d(_arr(q)), _d(p), C.POINTER(C.c_double)())
    return p


# ------------------------------------------------------------- SQP pieces

def cold_start(prob):
    """Reading c14: X_k = x_s for every knot, U = 0, nu = 0."""
    nx, nu = 2 * prob.model.dof, prob.model.dof
    X = np.tile(_arr(prob.x_s), (prob.N + 1, 1))
    U = np.zeros((prob.N, nu))
    lam = np.zeros((prob.N + 1, nx))
    return X, U, lam


def linearize(prob, X, U):
    P = _Prob(prob)
    N, nx, nu = P.N, P.nx, P.nu
    out = dict(A=np.zeros((N, nx, nx)), B=np.zeros((N, nx, nu)), Q=np.zeros((N + 1, nx, nx)),
               R=np.zeros((N, nu, nu)), q=np.zeros((N + 1, nx)), r=np.zeros((N, nu)),
               c=np.zeros((N + 1, nx)))
    X, U = _arr(X), _arr(U)
    J = lib().ora_linearize(C.byref(P.model), C.byref(P.p), _d(X), _d(U), _d(out["A"]),
                            _d(out["B"]), _d(out["Q"]), _d(out["R"]), _d(out["q"]),
                            _d(out["r"]), _d(out["c"]))
    out["J"] = J
    return out


def schur(prob, X, U, precond=0):
    P = _Prob(prob)
    N, nx = P.N, P.nx
    Sd = np.zeros((N + 1, nx, nx))
    Ss = np.zeros((N, nx, nx))
    Pd = np.zeros((N + 1, nx, nx))
    Ps = np.zeros((N, nx, nx))
    rhs = np.zeros((N + 1, nx))
    rc = lib().ora_schur(C.byref(P.model), C.byref(P.p), _d(_arr(X)), _d(_arr(U)), precond,
                         _d(Sd), _d(Ss), _d(Pd), _d(Ps), _d(rhs))
    if rc != 0:
        raise FloatingPointError("Schur blocks not positive definite")
    return dict(Sd=Sd, Ss=Ss, Pd=Pd, Ps=Ps, rhs=rhs)


def pcg(Sd, Ss, Pd, Ps, rhs, eps=1e-6, maxit=200, nu0=None):
    N = Sd.shape[0] - 1
    nx = Sd.shape[1]
    nu = np.zeros((N + 1, nx)) if nu0 is None else _arr(nu0).copy()
    it = lib().ora_pcg(N, nx, _d(_arr(Sd)), _d(_arr(Ss)), _d(_arr(Pd)), _d(_arr(Ps)),
                       _d(_arr(rhs)), eps, maxit, _d(nu))
    return nu, it


def blocktri_solve(Sd, Ss, rhs):
    N = Sd.shape[0] - 1
    nx = Sd.shape[1]
    x = np.zeros((N + 1, nx))
    rc = lib().ora_blocktri_solve(N, nx, _d(_arr(Sd)), _d(_arr(Ss)), _d(_arr(rhs)), _d(x))
    if rc != 0:
        raise FloatingPointError("block-tridiagonal factorisation failed")
    return x


def qp_step(prob, X, U, nu=None, precond=0, eps=1e-6, maxit=200):
    P = _Prob(prob)
    N, nx, nuu = P.N, P.nx, P.nu
    lam = np.zeros((N + 1, nx)) if nu is None else _arr(nu).copy()
    dX = np.zeros((N + 1, nx))
    dU = np.zeros((N, nuu))
    it = lib().ora_qp_step(C.byref(P.model), C.byref(P.p), _d(_arr(X)), _d(_arr(U)), precond,
                           eps, maxit, _d(lam), _d(dX), _d(dU))
    if it < 0:
        raise FloatingPointError("QP step failed")
    return dX, dU, lam, it


def merit(prob, X, U, mu=10.0):
    P = _Prob(prob)
    return lib().ora_merit(C.byref(P.model), C.byref(P.p), _d(_arr(X)), _d(_arr(U)), mu)


def kkt_residual(prob, X, U, nu):
    P = _Prob(prob)
    return lib().ora_kkt_residual(C.byref(P.model), C.byref(P.p), _d(_arr(X)), _d(_arr(U)),
                                  _d(_arr(nu)))


DEFAULTS = dict(mu=10.0, beta=2.0, n_alpha=8, pcg_eps=1e-6, pcg_max=1000, precond=0,
                kkt_tol=0.0, max_iter=10, linsolve=0, rho_adapt=0)


def solve(prob, max_iter=10, X=None, U=None, lam=None, replay=None, **kw):
    """Full SQP solve in FP64.  Returns a dict with the final iterate and logs."""
    P = _Prob(prob)
    prm = dict(DEFAULTS)
    prm.update(kw)
    prm["max_iter"] = max_iter
    params = OraParams(**prm)
    X0, U0, L0 = cold_start(prob)
    X = X0 if X is None else _arr(X).copy()
    U = U0 if U is None else _arr(U).copy()
    lam = L0 if lam is None else _arr(lam).copy()
    n = max(1, max_iter)
    la = np.full(n, -2, np.int32)
    lp = np.zeros(n, np.int32)
    m0, m1, kk, gap = (np.full(n, np.nan) for _ in range(4))
    rp = None if replay is None else np.ascontiguousarray(np.asarray(replay, np.int32))
    res = OraResult()
    lib().ora_solve(C.byref(P.model), C.byref(P.p), C.byref(params), _d(X), _d(U), _d(lam),
                    _i(rp) if rp is not None else C.POINTER(C.c_int32)(), _i(la), _i(lp),
                    _d(m0), _d(m1), _d(kk), _d(gap), C.byref(res))
    k = res.iters
    return dict(X=X, U=U, lam=lam, iters=res.iters, flags=res.flags, pcg_total=res.pcg_total,
                kkt=res.kkt, merit=res.merit, alpha_idx=la[:k].copy(), pcg_iters=lp[:k].copy(),
                merit_before=m0[:k].copy(), merit_after=m1[:k].copy(), kkt_log=kk[:k].copy(),
                merit_gap=gap[:k].copy())


FLOP_PRIMITIVES = ("rnea", "rnea_tangent_and_value", "cholesky_solve", "fk", "fk_and_tangent",
                   "block_product_14", "blocktri_row_14", "forward_dynamics")


def count_flops(model):
    """Operation counts (FMA = 2) of the method's primitive computations for
    `model`, from the oracle's formulas run on a FLOP-counting scalar: a dict
    keyed by FLOP_PRIMITIVES (see ora_count_flops in gato_oracle.cpp)."""
    m = make_model(model)
    return {name: int(lib().ora_count_flops(C.byref(m), i)) for i, name in enumerate(FLOP_PRIMITIVES)}
