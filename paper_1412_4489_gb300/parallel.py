"""Ranks of a multi-GPU run (one process per GPU, launched by torch.distributed.run).

The scheme's grids are independent problems, so a batch shards across ranks with no
exchange on the data path: each rank advances its own share of the grids, and the only
collectives are the scalar reductions of the measurement (total cells, slowest rank).
A single grid is not partitioned: each rank runs its own replica.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment; (0, 1, 0) alone."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_grids(cells: list[int], world: int) -> list[list[int]]:
    """Indices of the grids each rank advances: largest grid first onto the rank with the
    fewest cells so far (ties to the lowest rank), so shares differ by at most one grid's
    cells.  Deterministic: every rank computes the same assignment."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    shards: list[list[int]] = [[] for _ in range(world)]
    for g in sorted(range(len(cells)), key=lambda k: (-cells[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        shards[r].append(g)
        load[r] += cells[g]
    return [sorted(s) for s in shards]


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """The largest value over ranks (the slowest rank's time); x itself when alone."""
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device=None) -> float:
    """The sum over ranks (total cells advanced); x itself when alone."""
    return _reduce(x, "sum", device)
