"""gato_solve_noalloc: the solve entry point for callers that cannot allocate.

It runs the same kernel as gato_solve with its scratch in fixed arrays inside
the library.  The launch plan (latency form, one cluster size per horizon,
the same order) and every solve's arithmetic are the same as gato_solve's
automatic choice; only where the workspace lives differs.  So on the same
inputs its output must equal gato_solve's bit for bit, for the default
solver (PCG), the direct linear solve and rho adaptation alike, on two calls in
a row (the second reuses the scratch the first left behind), and through an
escalation to the high-precision mode.  This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_07625_gb300 import build, gato

    build.build_library()
    gato.load()
    return gato


def _results(dev):
    raw = dev.cpu().numpy()
    ints = raw.view(np.int32).reshape(-1, 5)
    flts = raw.view(np.float32).reshape(-1, 5)
    return ints[:, :3], flts[:, 3:]


def _run_pair(G, probs, iters, **prm):
    import torch

    models = [I.arm7(), I.arm6()]
    ref = G.Batch(models, len(probs), max(p.N for p in probs), **prm)
    a = G.DeviceProblems(ref, probs)
    res_ref = ref.solve(a.arr, a.n, iters)
    torch.cuda.synchronize()
    b = G.DeviceProblems(ref, probs)  # same inputs, separate buffers
    md = (G.ModelDesc * 2)(*[G.model_desc(m) for m in models])
    out = torch.zeros(len(probs) * 5, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    params = G.gato_default_params()
    for k, v in prm.items():
        setattr(params, k, v)
    G.gato_solve_noalloc(md, 2, params, b.arr, b.n, iters, out.data_ptr(), stream)
    torch.cuda.synchronize()
    ints, flts = _results(out)
    for i in range(len(probs)):
        Xa, Ua, La = a.solution(i)
        Xb, Ub, Lb = b.solution(i)
        for x, y in ((Xa, Xb), (Ua, Ub), (La, Lb)):
            np.testing.assert_array_equal(y, x)
        assert tuple(ints[i]) == (res_ref[i].flags, res_ref[i].sqp_iters, res_ref[i].pcg_iters)
        np.testing.assert_array_equal(flts[i], np.float32([res_ref[i].kkt_residual, res_ref[i].merit]))
    ref.close()


@pytest.mark.parametrize("prm", [{}, {"linsolve": 1}, {"rho_adapt": 1}],
                         ids=["pcg", "direct", "rho_adapt"])
def test_noalloc_matches_gato_solve_two_calls(G, prm):
    first = [I.joint_problem(s, I.arm7(), 32, 0.01) for s in range(5)] + [I.joint_problem(5, I.arm6(), 20)]
    _run_pair(G, first, 4, **prm)
    second = [I.ee_problem(s, I.arm7(), 64, 0.01) for s in range(3)] + [I.joint_problem(7, I.arm7(), 48)]
    _run_pair(G, second, 3, **prm)


def test_noalloc_matches_gato_solve_through_escalation(G):
    """With a KKT tolerance the solves escalate to the high-precision mode:
    the FP32 kernel leaves a hand-over record in the solve's workspace and the
    high-precision kernel resumes it.  Through the static scratch the records
    and the resumed solves must equal gato_solve's bit for bit."""
    from tests.test_gpu_parity import gpu_solve

    # a tolerance below the FP32 floor: the solves escalate and go on
    # iterating in the mode (so the log shows it)
    probs = [I.joint_problem(3, I.arm7(), N=12), I.joint_problem(1, I.arm7(), 32, 0.01),
             I.joint_problem(5, I.arm6(), 20)]
    logged = gpu_solve(G, probs, 30, log=True, kkt_tol=1e-9)
    assert sum(bool(r["hp"].any()) for r in logged) >= 1, "no solve escalated"
    _run_pair(G, probs, 30, kkt_tol=1e-9)


def test_noalloc_rejects_sizes_beyond_its_limits(G):
    import torch

    probs = [I.joint_problem(0, I.arm7(), 80, 0.01)]
    B = G.Batch([I.arm7()], 1, 80)
    dp = G.DeviceProblems(B, probs)
    md = (G.ModelDesc * 1)(G.model_desc(I.arm7()))
    out = torch.zeros(5, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GatoError) as e:
        G.gato_solve_noalloc(md, 1, G.gato_default_params(), dp.arr, 1, 2, out.data_ptr())
    assert e.value.status == G.GATO_E_INVALID
    many = [I.joint_problem(s, I.arm7(), 8, 0.01) for s in range(17)]
    B2 = G.Batch([I.arm7()], 17, 8)
    dp2 = G.DeviceProblems(B2, many)
    out2 = torch.zeros(17 * 5, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GatoError):
        G.gato_solve_noalloc(md, 1, G.gato_default_params(), dp2.arr, 17, 2, out2.data_ptr())
    B.close()
    B2.close()
