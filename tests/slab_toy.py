"""A host-side stand-in for a slab of the partitioned step, for testing the decomposition's
orchestration on CPU: it has the same phases and edge rows as a gks slab (CFL bound,
reconstruction, record exchange, faces and update, state exchange) around a small explicit
stencil that is asymmetric in y, so that a halo routed to the wrong side, a wrong neighbour
or a dt not reduced over all slabs changes the result.  Not the scheme: test infrastructure."""
import numpy as np
import torch

LOW, HIGH, STATE, RECORDS, EXCHANGE = 2, 3, 0, 1, 5


class ToySlab:
    def __init__(self, problem, precision=None, **opts):
        self.nx, self.ny = problem.nx, problem.ny
        self.kind = [b[0] for b in problem.bc]
        self.q = np.zeros((self.ny + 2, self.nx))  # rows -1 .. ny
        self.q[1:-1] = problem.U[0] + 0.1 * problem.U[3]
        self.r = np.zeros_like(self.q)
        self.t = 0.0
        self._wall(self.q)

    def _wall(self, a):
        # the grid's own y-boundaries: outflow (the edge row continued)
        if self.kind[2] != EXCHANGE and self.kind[2] != 0:
            a[0] = a[1]
        if self.kind[3] != EXCHANGE and self.kind[3] != 0:
            a[-1] = a[-2]

    def bound(self):
        return float(np.min(1.0 / (1.0 + np.abs(self.q[1:-1]))))

    def recon(self, dt):
        self.dt = dt
        q = self.q
        self.r[1:-1] = q[1:-1] + 0.3 * q[2:] - 0.2 * q[:-2] + 0.05 * np.roll(q[1:-1], 1, axis=1)
        self._wall(self.r)

    def finish(self):
        r, dt = self.r, self.dt
        F = 0.6 * r[:-1] + 0.4 * r[1:]  # face between rows k-1 and k (k = 0 .. ny)
        G = 0.7 * r[1:-1] + 0.3 * np.roll(r[1:-1], -1, axis=1)
        self.q[1:-1] = self.q[1:-1] - dt * (F[1:] - F[:-1]) - dt * (G - np.roll(G, 1, axis=1))
        self._wall(self.q)
        self.t += dt

    def edge(self, side, what):
        a = self.q if what == STATE else self.r
        row = a[1] if side == LOW else a[-2]
        return torch.from_numpy(np.ascontiguousarray(row).view(np.uint8).copy())

    def set_halo(self, side, what, buf):
        a = self.q if what == STATE else self.r
        row = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=np.float64)
        if side == LOW:
            a[0] = row
        else:
            a[-1] = row

    def state(self):
        return self.q[1:-1].copy(), self.t

    def close(self):
        pass
