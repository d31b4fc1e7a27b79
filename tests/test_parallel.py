"""The multi-rank host logic on CPU: grid sharding of a batch across ranks (each grid on
exactly one rank, balanced cell counts) and the measurement's reductions, with the gloo
backend at world size 2 and 3 (the GPU runs use NCCL with the same calls)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
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


# ---------------- domain decomposition of one grid into row slabs ----------------

def _toy_problem(periodic, ny=13, nx=7):
    from paper_1412_4489_gb300.workloads import Problem
    import numpy as np
    rng = np.random.default_rng(3)
    kind = 0 if periodic else 1
    bc = [(0, 0.0, 0.0, 1.0)] * 2 + [(kind, 0.0, 0.0, 1.0)] * 2
    U = 0.2 * rng.standard_normal((4, ny, nx))
    return Problem("toy", nx, ny, 1.0, 1.3, 1.4, 0.0, 1.0, bc, U, np.zeros((4, 2, ny, nx + 1)),
                   np.zeros((4, 2, ny + 1, nx)))


def _toy_run(problem, nslabs, steps):
    from slab_toy import ToySlab
    run = parallel.LocalSlabs(problem, nslabs, None, engine=ToySlab)
    for _ in range(steps):
        run.step(0.4)
    import numpy as np
    out = np.concatenate([s.state()[0] for s in run.slabs], axis=0)
    return out


def test_slab_rows_and_neighbours():
    for ny in (1, 5, 13, 64):
        for n in range(1, min(ny, 6) + 1):
            rows = parallel.slab_rows(ny, n)
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            h = [j1 - j0 for j0, j1 in rows]
            assert min(h) >= 1 and max(h) - min(h) <= 1
    assert parallel.slab_neighbours(0, 3, False) == (None, 1)
    assert parallel.slab_neighbours(2, 3, False) == (1, None)
    assert parallel.slab_neighbours(0, 3, True) == (2, 1)
    assert parallel.slab_neighbours(0, 1, True) == (0, 0)
    with pytest.raises(ValueError):
        parallel.slab_rows(3, 4)


@pytest.mark.parametrize("n", [32, 36])
def test_slab_problem_reproduces_the_cell_size(n):
    """A slab's height reproduces the grid's cell size exactly when a float height reaches it
    (every power-of-two cell size: n = 32), else to one ulp (n = 36: no float L has L / 7 equal
    to the float 1/36)."""
    import math
    p = wl.cavity_2d(n)
    dy = p.Ly / p.ny
    for j0, j1 in parallel.slab_rows(n, 5):
        s = parallel.slab_problem(p, j0, j1, 0 if j0 > 0 else None, 0 if j1 < n else None)
        if n == 32:
            assert s.Ly / s.ny == dy
        else:
            assert abs(s.Ly / s.ny - dy) <= math.ulp(dy)
        assert s.Wy.shape[2] == j1 - j0 + 1 and (s.Wy == p.Wy[:, :, j0:j1 + 1]).all()
        assert s.bc[2][0] == (5 if j0 > 0 else p.bc[2][0]) and s.bc[3][0] == (5 if j1 < n else p.bc[3][0])


@pytest.mark.parametrize("periodic", [True, False])
def test_local_slabs_equal_the_single_slab_bitwise(periodic):
    p = _toy_problem(periodic)
    ref = _toy_run(p, 1, 12)
    for n in (2, 3, 5):
        assert (_toy_run(p, n, 12) == ref).all(), n


def _slab_worker(rank, world, port, periodic, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from slab_toy import ToySlab
        run = parallel.DistributedSlab(_toy_problem(periodic), None, engine=ToySlab)
        dts = [run.step(0.4) for _ in range(12)]
        q.put((rank, run.state()[0], dts))
        run.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True)])
def test_distributed_slabs_equal_the_single_slab_bitwise(world, periodic):
    """Each gloo rank advances one slab; edges travel by point-to-point messages and the dt
    is a min-reduction over the ranks.  Joined in rank order the slabs equal the one-slab run
    bit for bit (two ranks on a periodic axis are each other's neighbour on both sides)."""
    import numpy as np
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, periodic, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted([q.get(timeout=120) for _ in range(world)], key=lambda o: o[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    got = np.concatenate([o[1] for o in out], axis=0)
    assert all(o[2] == out[0][2] for o in out)  # every rank took the same dt
    assert (got == _toy_run(_toy_problem(periodic), 1, 12)).all()
