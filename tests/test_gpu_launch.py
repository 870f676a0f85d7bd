"""Launch configurations, the autotuner and CUDA graph capture (GPU).

Every configuration runs the same arithmetic per knot; they differ in how the
knots of a solve are spread over CTAs and where the PCG's block rows live.
The two kernel forms with the same partition must agree bit for bit; other
partitions change only the order of the cluster-wide sums, so they are held to
the per-step parity bound against the oracle (Sec. III-B's M-block mapping).
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I
from tests.test_gpu_parity import _per_step_parity, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2510_07625_gb300 import gato
    gato.load()
    return gato


def test_throughput_form_equals_latency_form_bitwise(G):
    probs = [I.ee_problem(0, I.arm7(), 64), I.joint_problem(1, I.arm7(), 32, 0.01),
             I.joint_problem(2, I.arm6(), 100, 0.01)]
    a = gpu_solve(G, probs, 3, launch=(1, 0, 0))
    b = gpu_solve(G, probs, 3, launch=(2, 0, 0))
    for x, y in zip(a, b):
        for k in ("X", "U", "lam"):
            np.testing.assert_array_equal(x[k], y[k])
        assert (x["flags"], x["sqp_iters"], x["pcg_iters"]) == (y["flags"], y["sqp_iters"], y["pcg_iters"])


@pytest.mark.parametrize("launch", [(1, 9, 0), (2, 12, 0), (0, 0, 4), (0, 6, 0)],
                         ids=["lat-kpc9", "thr-kpc12", "uniform4", "kpc6"])
def test_spread_partitions_per_step_parity(G, oracle, launch):
    _per_step_parity(G, oracle, I.ee_problem(3, I.arm7(), 48, 0.01), 3, launch=launch)


def test_spread_partition_same_iteration_counts_early(G):
    # one SQP step from the cold start: the partition changes sums only in the
    # last bits, so the step lands within FP32 noise of the default partition
    p = I.joint_problem(4, I.arm7(), 64, 0.01)
    a = gpu_solve(G, [p], 1)[0]
    b = gpu_solve(G, [p], 1, launch=(0, 9, 0))[0]
    assert np.abs(a["X"] - b["X"]).max() <= 1e-4 * max(1.0, np.abs(a["X"]).max())


def test_autotune_leaves_iterates_and_matches_forced(G):
    import torch

    probs = [I.ee_problem(s, I.arm7(), 40) for s in range(6)]
    B = G.Batch([I.arm7()], len(probs), 40)
    dp = G.DeviceProblems(B, probs)
    X0, U0 = dp.X.clone(), dp.U.clone()
    cfg, ms = B.autotune(dp.arr, dp.n, 2, reps=1)
    torch.cuda.synchronize()
    assert cfg["variant"] in (1, 2) and ms > 0
    assert torch.equal(dp.X, X0) and torch.equal(dp.U, U0)
    # the tuned choice is used for this batch-size / horizon bucket
    r1 = B.solve(dp.arr, dp.n, 2)
    torch.cuda.synchronize()
    X1 = dp.X.clone()
    dp.reset()
    B.set_launch_config(cfg["variant"], cfg["knots_per_cta"], cfg["cluster"])
    r2 = B.solve(dp.arr, dp.n, 2)
    torch.cuda.synchronize()
    assert torch.equal(dp.X, X1)
    assert [r1[i].pcg_iters for i in range(dp.n)] == [r2[i].pcg_iters for i in range(dp.n)]
    B.close()


def test_launch_config_rejects_out_of_range(G):
    B = G.Batch([I.arm7()], 1, 8)
    for bad in [(3, 0, 0), (0, 1, 0), (0, 40, 0), (0, 0, 9)]:
        with pytest.raises(G.GatoError) as e:
            B.set_launch_config(*bad)
        assert e.value.status == G.GATO_E_INVALID
    B.close()


@pytest.mark.parametrize("launch", [None, (0, 0, 4)], ids=["grouped", "one-launch"])
def test_graph_replay_equals_solve(G, launch):
    """The uneven mix (two arms, N in 16..128, per-solve stop at KKT 1e-5 or 20
    iterations) captured in a CUDA graph: each replay equals gato_solve."""
    import torch

    probs = I.config_uneven(B=12)
    models = [I.arm7(), I.arm6()]
    B = G.Batch(models, len(probs), 128, kkt_tol=1e-5)
    if launch:
        B.set_launch_config(*launch)
    dp = G.DeviceProblems(B, probs)
    ref = B.solve(dp.arr, dp.n, 20)
    torch.cuda.synchronize()
    X_ref, U_ref = dp.X.clone(), dp.U.clone()
    dp.reset()
    gr = B.capture(dp.arr, dp.n, 20)
    for _ in range(2):
        dp.reset()
        torch.cuda.synchronize()
        res = gr.replay()
        assert torch.equal(dp.X, X_ref) and torch.equal(dp.U, U_ref)
        for i in range(dp.n):
            assert (res[i].flags, res[i].sqp_iters, res[i].pcg_iters) == \
                (ref[i].flags, ref[i].sqp_iters, ref[i].pcg_iters)
    gr.close()
    B.close()


def test_graph_rejects_host_problems(G):
    p = I.joint_problem(0, I.arm7(), 8, 0.01)
    B = G.Batch([I.arm7()], 1, 8)
    hp = G.HostProblems(B, [p])
    with pytest.raises(G.GatoError) as e:
        B.capture(hp.arr, 1, 2)
    assert e.value.status == G.GATO_E_INVALID
    B.close()


def test_query_launch_shapes(G):
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    a = G.gato_query_launch(32, 1)
    assert (a["ctas_per_solve"], a["variant"]) == (1, 1)
    assert 1 <= a["max_resident_solves"] <= sms
    b = G.gato_query_launch(64, 256)
    assert b["ctas_per_solve"] == 2 and b["variant"] in (1, 2)
    assert 1 <= b["max_resident_solves"] <= sms * 2 // 2
    c = G.gato_query_launch(64, 4, variant=1, knots_per_cta=9)
    assert c["ctas_per_solve"] == 8 and c["variant"] == 1
    assert c["max_resident_solves"] <= sms // 8
    d = G.gato_query_launch(64, 4, variant=2)
    assert d["variant"] == 2 and d["smem_bytes"] == b["smem_bytes"]
    # two CTAs per SM in the throughput form: at least as many resident solves
    assert d["max_resident_solves"] >= G.gato_query_launch(64, 4, variant=1)["max_resident_solves"]
    with pytest.raises(G.GatoError):
        G.gato_query_launch(0, 1)
    with pytest.raises(G.GatoError):
        G.gato_query_launch(300, 1)


# (N, uniform cluster) -> CTA knot counts: (9, 4) -> 3,3,3,1; (7, 4) -> 2,2,2,2;
# (6, 3) -> 3,3,1; (24, 8) -> 4 x 6, 1; (64, 8) -> 9 x 7, 2; (64, 2) -> 33, 32;
# (98, 3) -> 33 x 3, (128, 4) -> 33, 33, 33, 30 and (256, 8) -> 33 x 7, 26: middle
# CTAs of 30 or more knots, whose fourth halo knot sits on the last warp (the
# others on spare lanes); CTAs of at most 29 knots keep all halo knots on one
# free warp
HALO_CASES = [(9, 4), (7, 4), (6, 3), (24, 8), (64, 8), (64, 2), (98, 3), (128, 4), (256, 8)]


@pytest.mark.parametrize("precond", [0, 1], ids=["stair", "jacobi"])
@pytest.mark.parametrize("N,cl", HALO_CASES, ids=[f"N{n}-C{c}" for n, c in HALO_CASES])
def test_halo_recompute_equals_pushed_halos_bitwise(G, N, cl, precond):
    # The latency form recomputes the neighbours' halo knots inside each CTA;
    # the throughput form exchanges y and u rows through distributed shared
    # memory.  Both must give the same bits, including CTAs with one or two
    # knots (whose halo knots reach the neighbour's first or last knot).
    probs = [I.ee_problem(7, I.arm7(), N), I.joint_problem(8, I.arm7(), N, 0.01),
             I.joint_problem(9, I.arm6(), N, 0.01)]
    a = gpu_solve(G, probs, 3, launch=(1, 0, cl), precond=precond)
    b = gpu_solve(G, probs, 3, launch=(2, 0, cl), precond=precond)
    for x, y in zip(a, b):
        for k in ("X", "U", "lam"):
            np.testing.assert_array_equal(x[k], y[k])
        assert (x["flags"], x["sqp_iters"], x["pcg_iters"]) == (y["flags"], y["sqp_iters"], y["pcg_iters"])


@pytest.mark.parametrize("N", [64, 100])
def test_halo_recompute_equals_plain_exchange_bitwise(G, N):
    # The plain form, like the throughput form, exchanges boundary y and u
    # rows between the CTAs of a cluster; the fused latency form, with the
    # same split of the knots (cluster_for(N) CTAs), recomputes them.  Two
    # and four CTAs.
    probs = [I.ee_problem(7, I.arm7(), N), I.joint_problem(9, I.arm6(), N, 0.01)]
    for p in probs:
        a = gpu_solve(G, [p], 3, launch=(1, 0, 0))[0]
        b = gpu_solve(G, [p], 3, plain=True)[0]
        for k in ("X", "U", "lam"):
            np.testing.assert_array_equal(a[k], b[k])
        assert (a["flags"], a["sqp_iters"], a["pcg_iters"]) == (b["flags"], b["sqp_iters"], b["pcg_iters"])
