"""Splitting one list of solves over several GPUs (one process per GPU).

Solves are independent (Sec. III-B: no coordination between the blocks of
different solves), so a multi-GPU run needs no collective on the data path:
each rank takes its share, solves it with its own batch and keeps its
results; a host gather, if wanted, only collects them.  Shares are balanced
by knots (N + 1) with the longest-processing-time-first rule: solves in order
of decreasing knots, each to the rank with the fewest knots so far (ties:
lower index first, lower rank first), which stays within 4/3 of the best
split.
"""
from __future__ import annotations


def lpt_assign(costs, n_parts):
    """Index lists, one per part, from the LPT rule over `costs`."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * n_parts
    parts = [[] for _ in range(n_parts)]
    for i in order:
        r = min(range(n_parts), key=lambda p: (load[p], p))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def shard(problems, rank, world):
    """(indices, problems) of this rank's share, balanced by knots."""
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    idx = lpt_assign([p.N + 1 for p in problems], world)[rank]
    return idx, [problems[i] for i in idx]
