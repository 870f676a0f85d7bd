"""Multi-process path of bench.py on CPU (gloo, world_size 2).

Replicas solve disjoint seeded batches and only the timing is combined: the
whole-job rate divides every rank's solves by the slowest rank's time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench.dist_env()
        t = [1.5, 2.5][rank]  # this rank's timed seconds
        t_max = bench.max_over_ranks(t, "cpu")
        seeds = list(range(bench.rank_seed0(r, 4), bench.rank_seed0(r, 4) + 4))
        out[rank] = (w, t_max, bench.whole_job_rate(w, 4, 10, t_max), seeds)
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        w, t_max, rate, _ = res[rank]
        assert w == 2 and t_max == 2.5
        assert rate == pytest.approx(2 * 4 * 10 / 2.5)
    assert not set(res[0][3]) & set(res[1][3])  # disjoint problem seeds


def test_single_process_defaults():
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    assert bench.whole_job_rate(1, 256, 10, 2.0) == 1280.0
