"""The multi-rank host logic on CPU: grid sharding of a batch across ranks (each grid on
exactly one rank, balanced cell counts) and the measurement's reductions, with the gloo
backend at world size 2 and 3 (the GPU runs use NCCL with the same calls)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1412_4489_gb300 import parallel, workloads as wl


def test_shard_grids_covers_every_grid_once_and_balances():
    cells = [sp[0] * sp[1] for sp in wl.batch_specs(512, seed=5)]
    for world in (1, 2, 3, 8):
        shards = parallel.shard_grids(cells, world)
        flat = sorted(g for s in shards for g in s)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[g] for g in s) for s in shards]
        assert max(loads) - min(loads) <= max(cells)
    with pytest.raises(ValueError):
        parallel.shard_grids(cells, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cells, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = parallel.rank_env()
        mine = parallel.shard_grids(cells, w)[r]
        total = parallel.sum_over_ranks(sum(cells[g] for g in mine))
        slowest = parallel.max_over_ranks(1.0 + r)
        q.put((r, w, lr, mine, total, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_shard_the_batch_and_reduce(world):
    cells = [sp[0] * sp[1] for sp in wl.batch_specs(64, seed=5)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cells, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == list(range(world)) and all(o[1] == world for o in out)
    assert sorted(g for o in out for g in o[3]) == list(range(len(cells)))
    assert all(o[4] == sum(cells) for o in out)
    assert all(o[5] == float(world) for o in out)


def test_alone_the_reductions_are_identities():
    assert parallel.max_over_ranks(3.5) == 3.5
    assert parallel.sum_over_ranks(2.0) == 2.0
