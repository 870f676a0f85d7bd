"""Multi-GPU sharding of one problem list (replicas, no data-path collective):
the LPT split covers every solve exactly once, balances knots, and two gloo
ranks that each take their share gather back the whole list (CPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_07625_gb300 import inputs as I
from paper_2510_07625_gb300 import sharding


def test_lpt_split_covers_and_balances():
    probs = I.config_uneven(128)
    knots = [p.N + 1 for p in probs]
    for world in (1, 2, 3, 4, 8):
        parts = sharding.lpt_assign(knots, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(probs)))
        loads = [sum(knots[i] for i in p) for p in parts]
        # LPT: the heaviest part exceeds the mean by less than the largest job
        assert max(loads) - sum(loads) / world < max(knots)
        assert sharding.lpt_assign(knots, world) == parts  # deterministic
    with pytest.raises(ValueError):
        sharding.lpt_assign(knots, 0)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        probs = I.config_uneven(40)
        idx, mine = sharding.shard(probs, rank, ws)
        # each rank's "result": its solves' horizons; only the gather is collective
        t = torch.full((len(probs),), -1, dtype=torch.int64)
        for i, p in zip(idx, mine):
            t[i] = p.N
        got = [torch.empty_like(t) for _ in range(ws)]
        dist.all_gather(got, t)
        out[rank] = torch.stack(got).max(dim=0).values.tolist()
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_gather_the_whole_list():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(ws, _port(), out), nprocs=ws, join=True)
    want = [p.N for p in I.config_uneven(40)]
    assert out[0] == want and out[1] == want
