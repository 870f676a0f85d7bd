"""The closed-loop hypothesize-and-test run (Sec. IV-D) with the GPU batch
solve: a short run under an unmodelled end-effector force, latency fixed so
the run is reproducible.  The estimate approaches the force and the arm
stays on the track."""
import numpy as np
import pytest

from paper_2510_07625_gb300 import closed_loop as CL
from paper_2510_07625_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_gpu_closed_loop_estimates_the_force():
    from paper_2510_07625_gb300 import gato
    gato.load()
    model = I.arm6()
    plant = gato.Plant(model)
    f = np.array([0.0, 0.0, -50.0])
    solver = CL.GpuBatchSolver(model, 16, 32, 3)
    try:
        r = CL.run(solver, plant, 16, f, N=32, sim_s=0.3, latency_s=0.002, settle_s=0.1, radius=10.0)
    finally:
        solver.close()
    assert r.ticks == 150
    assert r.f_err < 0.5 * np.linalg.norm(f), r.f_est
    assert np.isfinite(r.track_err_mean) and r.track_err_mean < 0.5
