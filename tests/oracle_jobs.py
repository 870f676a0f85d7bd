"""Oracle runs farmed out to a process pool by the GPU parity tests.

Only the FP64 oracle runs here (test infrastructure).  The pool is started
with the spawn method, so no child inherits a CUDA context.
"""
from __future__ import annotations

import os

import numpy as np


def solve(args):
    """oracle.solve(prob, **kw) -> the dict it returns."""
    prob, kw = args
    import oracle

    return oracle.solve(prob, **kw)


def fixed_count_pair(args):
    """The oracle's iterate after `iters` SQP iterations twice: with PCG at its
    stopping tolerance (the method) and with the direct block elimination
    (the exact QP solution).  Their distance is how far the fixed-count
    iterate is determined by the method itself."""
    prob, iters, kw = args
    import oracle

    a = oracle.solve(prob, max_iter=iters, **kw)
    b = oracle.solve(prob, max_iter=iters, linsolve=1, **kw)
    spread = max(rel(a["X"], b["X"]), rel(a["U"], b["U"]))
    return a, spread


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1.0, np.abs(b).max()))


def pool():
    import multiprocessing as mp

    return mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
