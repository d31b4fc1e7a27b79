"""Ranks of a multi-GPU run (one process per GPU, launched by torch.distributed.run), and
the domain decomposition of one grid into row slabs.

Independent grids: a batch shards across ranks with no exchange on the data path; each rank
advances its own share of the grids, and the only collectives are the scalar reductions of
the measurement (total cells, slowest rank).

One grid: split into row slabs (the partitioned step of gks.h, Eq. finite over the whole
grid).  Each slab is a gks handle whose y-sides facing other slabs are exchange sides.  A
step is: the CFL bound's minimum over all slabs (the global dt), the reconstruction of every
slab, the exchange of the edge rows of reconstruction records, the face evolution and update
of every slab (both slabs evaluate a partition face from the same inputs), the exchange of
the edge rows of the new cell averages.  The slabs' states then equal the single-grid state
bit for bit.  LocalSlabs runs the slabs of one grid in one process (one GPU, host-ordered
exchanges, no kernel waits on another); DistributedSlab runs one slab per rank and exchanges
edges by point-to-point messages (NCCL between GPUs, gloo between host processes).
"""
from __future__ import annotations

import math
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


# ---------------------------------------------------------------------------
# domain decomposition of one grid into row slabs
# ---------------------------------------------------------------------------
LOW, HIGH = 2, 3        # y-sides of a slab (gks side numbering)
STATE, RECORDS = 0, 1   # what an edge row holds (GKS_PART_STATE, GKS_PART_RECORDS)
EXCHANGE = 5            # GKS_BC_EXCHANGE
PERIODIC = 0


def slab_rows(ny: int, nslabs: int) -> list[tuple[int, int]]:
    """Rows [j0, j1) of each slab: nslabs contiguous slabs whose heights differ by at most one."""
    if not 1 <= nslabs <= ny:
        raise ValueError("need 1 <= nslabs <= ny")
    base, extra = divmod(ny, nslabs)
    rows, j = [], 0
    for r in range(nslabs):
        h = base + (1 if r < extra else 0)
        rows.append((j, j + h))
        j += h
    return rows


def slab_neighbours(r: int, nslabs: int, periodic_y: bool) -> tuple[int | None, int | None]:
    """(slab below, slab above) of slab r, None where the grid ends (a periodic axis wraps)."""
    low = r - 1 if r > 0 else (nslabs - 1 if periodic_y else None)
    high = r + 1 if r < nslabs - 1 else (0 if periodic_y else None)
    return low, high


def _height_for(dy: float, n: int) -> float:
    """A slab height L whose cell size L / n is dy exactly where some L reaches it (every
    power-of-two dy, among others), so that the slab's constants equal the grid's bit for
    bit; else the L whose L / n is nearest (one ulp of dy off: the slabs then follow the
    single grid to roundoff, not bit for bit)."""
    L = dy * n
    best = L
    for _ in range(8):
        q = L / n
        if q == dy:
            return L
        if abs(q - dy) < abs(best / n - dy):
            best = L
        L = math.nextafter(L, math.inf if q < dy else -math.inf)
    return best


def slab_problem(p, j0: int, j1: int, low, high):
    """The problem of rows [j0, j1) of problem p: the rows of U and Wx, the rows j0..j1 of Wy
    (both partition faces), exchange sides where a neighbouring slab lies beyond."""
    from .workloads import Problem
    bc = list(p.bc)
    if low is not None:
        bc[2] = (EXCHANGE, 0.0, 0.0, 1.0)
    if high is not None:
        bc[3] = (EXCHANGE, 0.0, 0.0, 1.0)
    return Problem(f"{p.name}_rows_{j0}_{j1}", p.nx, j1 - j0, p.Lx, _height_for(p.Ly / p.ny, j1 - j0), p.gamma,
                   p.mu, p.Pr, bc, p.U[:, j0:j1].copy(), p.Wx[:, :, j0:j1].copy(), p.Wy[:, :, j0:j1 + 1].copy(),
                   p.CFL, dict(p.meta))


class GKSSlab:
    """One slab on this process's GPU: a gks handle with exchange sides.  Edge rows are
    returned in byte tensors on `device` (host memory for a host transport)."""

    def __init__(self, problem, precision, device="cuda", stream=None, **opts):
        import torch
        from . import gks
        self.gks = gks
        self.solver = gks.Solver(problem, precision, stream=stream, **opts)
        self.h = self.solver.h
        self.device = device
        self.nbytes = {w: gks.gks_part_halo_bytes(self.h, w) for w in (STATE, RECORDS)}
        self._torch = torch

    def bound(self) -> float:
        return self.gks.gks_part_bound(self.h)

    def recon(self, dt: float) -> None:
        self.gks.gks_part_recon(self.h, dt)

    def finish(self) -> None:
        self.gks.gks_part_finish(self.h)

    def edge(self, side: int, what: int):
        buf = self._torch.empty(self.nbytes[what], dtype=self._torch.uint8, device=self.device)
        self.gks.gks_part_get_edge(self.h, side, what, buf)
        return buf

    def set_halo(self, side: int, what: int, buf) -> None:
        self.gks.gks_part_set_halo(self.h, side, what, buf)

    def state(self):
        return self.solver.state()

    def close(self) -> None:
        self.solver.close()


def _join_states(states):
    """The grid's (U, Wx, Wy, t) from its slabs' states, in slab order (the partition faces'
    values are equal on both sides: the lower slab's copy is taken)."""
    import numpy as np
    U = np.concatenate([s[0] for s in states], axis=1)
    Wx = np.concatenate([s[1] for s in states], axis=2)
    Wy = np.concatenate([s[2][:, :, :-1] for s in states] + [states[-1][2][:, :, -1:]], axis=2)
    return U, Wx, Wy, states[0][3]


class LocalSlabs:
    """All slabs of one grid in this process: exchanges are copies ordered by the host."""

    def __init__(self, problem, nslabs, precision, engine=GKSSlab, **opts):
        periodic = problem.bc[2][0] == PERIODIC
        rows = slab_rows(problem.ny, nslabs)
        self.nbs = [slab_neighbours(r, nslabs, periodic) for r in range(nslabs)]
        self.slabs = [engine(slab_problem(problem, j0, j1, *self.nbs[r]), precision, **opts)
                      for r, (j0, j1) in enumerate(rows)]
        self.exchange(STATE)

    def exchange(self, what: int) -> None:
        # every edge first, then every halo (a slab can be its own neighbour)
        edges = [{side: s.edge(side, what) for side, nb in zip((LOW, HIGH), nb2) if nb is not None}
                 for s, nb2 in zip(self.slabs, self.nbs)]
        for r, (low, high) in enumerate(self.nbs):
            if low is not None:
                self.slabs[r].set_halo(LOW, what, edges[low][HIGH])
            if high is not None:
                self.slabs[r].set_halo(HIGH, what, edges[high][LOW])

    def step(self, CFL: float, dt_max: float = math.inf) -> float:
        dt = min(CFL * min(s.bound() for s in self.slabs), dt_max)
        for s in self.slabs:
            s.recon(dt)
        self.exchange(RECORDS)
        for s in self.slabs:
            s.finish()
        self.exchange(STATE)
        return dt

    def state(self):
        return _join_states([s.state() for s in self.slabs])

    def close(self) -> None:
        for s in self.slabs:
            s.close()


class DistributedSlab:
    """Slab `rank` of one grid split over the ranks of the default process group.  Edges
    travel by point-to-point messages: each rank sends its low edge to the slab below and its
    high edge to the slab above, and receives theirs into its halos; sends and receives are
    posted in an order that matches pairwise also when one neighbour lies on both sides (two
    slabs on a periodic axis).  The global dt is a min-reduction of the slabs' CFL bounds."""

    def __init__(self, problem, precision, engine=GKSSlab, comm_device="cpu", **opts):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        periodic = problem.bc[2][0] == PERIODIC
        j0, j1 = slab_rows(problem.ny, self.world)[self.rank]
        self.low, self.high = slab_neighbours(self.rank, self.world, periodic)
        self.comm_device = comm_device
        self.slab = engine(slab_problem(problem, j0, j1, self.low, self.high), precision, **opts)
        self.exchange(STATE)

    def exchange(self, what: int) -> None:
        import torch
        dist = self.dist
        out = {side: self.slab.edge(side, what) for side, nb in ((LOW, self.low), (HIGH, self.high)) if nb is not None}
        if self.world == 1:  # a single periodic slab is its own neighbour
            for side, src in ((LOW, HIGH), (HIGH, LOW)):
                if side in out:
                    self.slab.set_halo(side, what, out[src])
            return
        ops, inbox = [], {}
        if self.low is not None:
            ops.append(dist.P2POp(dist.isend, out[LOW].to(self.comm_device), self.low))
        if self.high is not None:
            ops.append(dist.P2POp(dist.isend, out[HIGH].to(self.comm_device), self.high))
        # a neighbour's sends arrive low edge first, then high edge: the high halo (its low
        # edge) is received first
        if self.high is not None:
            inbox[HIGH] = torch.empty_like(out[HIGH], device=self.comm_device)
            ops.append(dist.P2POp(dist.irecv, inbox[HIGH], self.high))
        if self.low is not None:
            inbox[LOW] = torch.empty_like(out[LOW], device=self.comm_device)
            ops.append(dist.P2POp(dist.irecv, inbox[LOW], self.low))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for side, buf in inbox.items():
            self.slab.set_halo(side, what, buf)

    def step(self, CFL: float, dt_max: float = math.inf) -> float:
        import torch
        b = torch.tensor([self.slab.bound()], dtype=torch.float64, device=self.comm_device)
        self.dist.all_reduce(b, op=self.dist.ReduceOp.MIN)
        dt = min(CFL * float(b.item()), dt_max)
        self.slab.recon(dt)
        self.exchange(RECORDS)
        self.slab.finish()
        self.exchange(STATE)
        return dt

    def state(self):
        return self.slab.state()

    def close(self) -> None:
        self.slab.close()
