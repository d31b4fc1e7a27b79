"""Seeded synthetic inputs shaped after the paper's test problems (Section 4).

This module holds only input generation: a SplitMix64 generator and the initial
cell averages and interface point values of each workload.  It contains none of the
scheme's arithmetic, so both the CUDA path and the oracle may use it.

Workloads (all FP64 host arrays in the library's SoA layout):

* ``density_wave_1d``  -- Section 4.1, rho = 1 + 0.2 sin(pi (x + phi)), U = 1, p = 1 on a
  periodic [0, 2] line, laid out as an nx-by-1 periodic 2D grid (dy = dx).
* ``smooth_wave_2d``   -- rho = 1 + 0.2 sin(pi (x + y) + phi), U = V = 1, p = 1 on the
  periodic square [0, 2]^2 (the 2D analogue of Section 4.1).
* ``riemann_2d``       -- four constant quadrants on [0, 1]^2 as in the 2D Riemann problems
  of Section 4, with seeded rho ~ U[0.1, 1.5], p ~ U[0.03, 1.5], u, v ~ U[-1, 1].
* ``cavity_2d``        -- lid-driven square cavity at rest (rho = 1, p = 1/gamma), lid speed
  0.15 (lid Mach number 0.15), isothermal no-slip walls.
* ``batch_grids``      -- 512 independent grids with seeded sizes, kinds, gamma and mu.
* ``isotropic_vortex`` -- Section 4.1's second accuracy test: an isentropic vortex of
  strength 5 on the mean flow (1, 1, 1, 1) in the periodic [-5, 5]^2 (Table 2).
* ``sod``              -- Section 4.2's Sod tube, (1, 0, 1) | (0.125, 0, 0.1) on [0, 1], as an
  nx-by-1 grid periodic in y with outflow ends.

Cell averages are exact averages of the initial data; interface values are the exact
point values at the Gauss points (x-faces: y_j -/+ sqrt(3)/6 dy; y-faces: x_i -/+ sqrt(3)/6 dx).
A point lying exactly on an initial discontinuity takes the mean of the two sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAUSS = math.sqrt(3.0) / 6.0


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014); doubles are (x >> 11) * 2^-53."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))


BC_PERIODIC, BC_OUTFLOW, BC_SLIPWALL, BC_NOSLIP_ISOTHERMAL, BC_NOSLIP_ADIABATIC = 0, 1, 2, 3, 4


@dataclass
class Problem:
    """A 2D grid problem: geometry, gas, boundary conditions and the initial state."""
    name: str
    nx: int
    ny: int
    Lx: float
    Ly: float
    gamma: float
    mu: float
    Pr: float
    bc: list  # 4 x (kind, u_wall, v_wall, T_wall): x-low, x-high, y-low, y-high
    U: np.ndarray   # [4][ny][nx]
    Wx: np.ndarray  # [4][2][ny][nx+1]
    Wy: np.ndarray  # [4][2][ny+1][nx]
    CFL: float = 0.5
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def _cons(rho, u, v, p, gamma):
    rho = np.asarray(rho, dtype=np.float64)
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def _gauss_points(nx, ny, Lx, Ly):
    dx, dy = Lx / nx, Ly / ny
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    xf = np.arange(nx + 1) * dx
    yf = np.arange(ny + 1) * dy
    # x-faces: (x = xf[i], y = yc[j] -/+ g dy)
    wx_pts = [(xf[None, :] + 0 * yc[:, None], yc[:, None] + s * GAUSS * dy + 0 * xf[None, :]) for s in (-1, 1)]
    wy_pts = [(xc[None, :] + s * GAUSS * dx + 0 * yf[:, None], yf[:, None] + 0 * xc[None, :]) for s in (-1, 1)]
    return xc, yc, wx_pts, wy_pts


def _point_state(fn, pts):
    return np.stack([fn(x, y) for (x, y) in pts], axis=1)  # [4][2][...]


def sinc(z):
    z = np.asarray(z, dtype=np.float64)
    return np.where(z == 0.0, 1.0, np.sin(z) / np.where(z == 0.0, 1.0, z))


def smooth_wave_2d(n: int, seed: int = 2, gamma: float = 1.4, L: float = 2.0, ny: int | None = None) -> Problem:
    """Periodic smooth wave rho = 1 + 0.2 sin(pi (x + y) + phi), U = V = 1, p = 1."""
    ny = n if ny is None else ny
    rng = SplitMix64(seed)
    phi = rng.uniform()
    nx = n
    Lx = Ly = L
    dx, dy = Lx / nx, Ly / ny
    xc, yc, wxp, wyp = _gauss_points(nx, ny, Lx, Ly)
    X, Y = np.meshgrid(xc, yc)
    rho_bar = 1.0 + 0.2 * np.sin(np.pi * (X + Y) + phi) * sinc(np.pi * dx / 2) * sinc(np.pi * dy / 2)
    U = np.stack([rho_bar, rho_bar, rho_bar, 1.0 / (gamma - 1.0) + rho_bar])

    def pt(x, y):
        r = 1.0 + 0.2 * np.sin(np.pi * (x + y) + phi)
        return _cons(r, 1.0, 1.0, 1.0, gamma)

    Wx = _point_state(pt, wxp)
    Wy = _point_state(pt, wyp)
    bc = [(BC_PERIODIC, 0.0, 0.0, 1.0)] * 4
    return Problem(f"smooth_wave_{nx}x{ny}", nx, ny, Lx, Ly, gamma, 0.0, 1.0, bc,
                   np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy),
                   meta={"phi": phi, "seed": seed})


def density_wave_1d(nx: int, seed: int = 1, gamma: float = 1.4, phi: float | None = None) -> Problem:
    """Section 4.1 density wave on [0, 2] as an nx-by-1 periodic grid with dy = dx."""
    if phi is None:
        phi = SplitMix64(seed).uniform()
    Lx = 2.0
    dx = Lx / nx
    Ly = dx
    xc, yc, wxp, wyp = _gauss_points(nx, 1, Lx, Ly)
    rho_bar = 1.0 + 0.2 * np.sin(np.pi * (xc + phi)) * sinc(np.pi * dx / 2)
    U = np.stack([rho_bar, rho_bar, 0 * rho_bar, 1.0 / (gamma - 1.0) + 0.5 * rho_bar])[:, None, :]

    def pt(x, y):
        r = 1.0 + 0.2 * np.sin(np.pi * (x + phi))
        return _cons(r, 1.0, 0.0, 1.0, gamma)

    Wx = _point_state(pt, wxp)
    Wy = _point_state(pt, wyp)
    bc = [(BC_PERIODIC, 0.0, 0.0, 1.0)] * 4
    return Problem(f"density_wave_{nx}", nx, 1, Lx, Ly, gamma, 0.0, 1.0, bc,
                   np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy),
                   meta={"phi": phi, "seed": seed})


def density_wave_exact_avg(nx: int, t: float, phi: float, gamma: float = 1.4):
    """Exact cell averages of rho at time t for the translated density wave."""
    dx = 2.0 / nx
    xc = (np.arange(nx) + 0.5) * dx
    return 1.0 + 0.2 * np.sin(np.pi * (xc - t + phi)) * sinc(np.pi * dx / 2)


def density_wave_1d_layout(p: Problem):
    """The same data in the 3-variable 1D layout U[3][nx], W[3][nx+1] (face-centre values)."""
    U1 = np.ascontiguousarray(np.stack([p.U[0, 0], p.U[1, 0], p.U[3, 0]]))
    # 1D face values are the point values at the face; with no y dependence both Gauss
    # points carry the same value
    W1 = np.ascontiguousarray(np.stack([p.Wx[0, 0, 0], p.Wx[1, 0, 0], p.Wx[3, 0, 0]]))
    return U1, W1


def riemann_draw(rng: SplitMix64):
    """Quadrant states in the order NE, NW, SW, SE; per quadrant rho, p, u, v."""
    q = []
    for _ in range(4):
        rho = rng.uniform(0.1, 1.5)
        p = rng.uniform(0.03, 1.5)
        u = rng.uniform(-1.0, 1.0)
        v = rng.uniform(-1.0, 1.0)
        q.append((rho, u, v, p))
    return q


def riemann_2d(nx: int, ny: int | None = None, seed: int = 3, gamma: float = 1.4, mu: float = 1e-4,
               Pr: float = 0.72, quadrants=None) -> Problem:
    """Four-quadrant Riemann data on [0, 1]^2 with outflow boundaries."""
    ny = nx if ny is None else ny
    if quadrants is None:
        quadrants = riemann_draw(SplitMix64(seed))
    Lx = Ly = 1.0
    dx, dy = Lx / nx, Ly / ny
    qs = [_cons(r, u, v, p, gamma) for (r, u, v, p) in quadrants]  # NE, NW, SW, SE

    def state_at(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros((4,) + np.broadcast(x, y).shape)
        east = np.where(x > 0.5, 1.0, np.where(x < 0.5, 0.0, 0.5))
        north = np.where(y > 0.5, 1.0, np.where(y < 0.5, 0.0, 0.5))
        w = [east * north, (1 - east) * north, (1 - east) * (1 - north), east * (1 - north)]
        for k in range(4):
            out += w[k][None] * qs[k].reshape(4, *([1] * x.ndim))
        return out

    # exact cell averages: area fractions of each quadrant
    xl = np.arange(nx) * dx
    yl = np.arange(ny) * dy
    fe = np.clip((xl + dx - 0.5) / dx, 0.0, 1.0)  # fraction of the cell east of x = 0.5
    fn = np.clip((yl + dy - 0.5) / dy, 0.0, 1.0)
    FE, FN = np.meshgrid(fe, fn)
    U = (qs[0].reshape(4, 1, 1) * FE * FN + qs[1].reshape(4, 1, 1) * (1 - FE) * FN +
         qs[2].reshape(4, 1, 1) * (1 - FE) * (1 - FN) + qs[3].reshape(4, 1, 1) * FE * (1 - FN))
    _, _, wxp, wyp = _gauss_points(nx, ny, Lx, Ly)
    Wx = _point_state(state_at, wxp)
    Wy = _point_state(state_at, wyp)
    bc = [(BC_OUTFLOW, 0.0, 0.0, 1.0)] * 4
    return Problem(f"riemann_{nx}x{ny}", nx, ny, Lx, Ly, gamma, mu, Pr, bc,
                   np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy),
                   meta={"quadrants": quadrants, "seed": seed})


def cavity_2d(n: int, gamma: float = 1.4, Re: float = 1000.0, lid: float = 0.15, Pr: float = 0.72) -> Problem:
    """Lid-driven square cavity, rho = 1, p = 1/gamma (sound speed 1), at rest."""
    nx = ny = n
    Lx = Ly = 1.0
    mu = 1.0 * lid * Lx / Re
    Tw = 1.0 / gamma
    U = np.ascontiguousarray(np.broadcast_to(_cons(1.0, 0.0, 0.0, 1.0 / gamma, gamma).reshape(4, 1, 1),
                                             (4, ny, nx)).copy())
    Wx = np.ascontiguousarray(np.broadcast_to(U[:, None, :, :1], (4, 2, ny, nx + 1)).copy())
    Wy = np.ascontiguousarray(np.broadcast_to(U[:, None, :1, :], (4, 2, ny + 1, nx)).copy())
    wall = (BC_NOSLIP_ISOTHERMAL, 0.0, 0.0, Tw)
    bc = [wall, wall, wall, (BC_NOSLIP_ISOTHERMAL, lid, 0.0, Tw)]
    return Problem(f"cavity_{n}", nx, ny, Lx, Ly, gamma, mu, Pr, bc, U, Wx, Wy,
                   meta={"Re": Re, "lid": lid})


def isotropic_vortex_state(x, y, gamma: float = 1.4, eps: float = 5.0):
    """Point state of the isotropic vortex centred at the origin on the mean flow
    (rho, u, v, p) = (1, 1, 1, 1): du, dv = eps/(2 pi) e^((1 - r^2)/2) (-y, x),
    dT = -(gamma - 1) eps^2 / (8 gamma pi^2) e^(1 - r^2), entropy p / rho^gamma = 1."""
    r2 = x * x + y * y
    f = eps / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi * np.pi) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    return _cons(rho, 1.0 - f * y, 1.0 + f * x, rho * T, gamma)


def _gl(nq: int):
    z, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * z, 0.5 * w  # nodes on [-1/2, 1/2], weights summing to 1


def isotropic_vortex(n: int, gamma: float = 1.4, eps: float = 5.0, nq: int = 6) -> Problem:
    """The vortex at the centre of the periodic square [-5, 5]^2 (grid origin at its corner),
    n x n cells.  Cell averages by an nq x nq Gauss-Legendre rule per cell; the face values
    are the exact point values at the Gauss points."""
    L = 10.0
    dx = dy = L / n
    xc = -5.0 + (np.arange(n) + 0.5) * dx
    z, w = _gl(nq)
    U = np.zeros((4, n, n))
    for a in range(nq):
        for b in range(nq):
            X, Y = np.meshgrid(xc + z[a] * dx, xc + z[b] * dy)
            U += w[a] * w[b] * isotropic_vortex_state(X, Y, gamma, eps)
    _, _, wxp, wyp = _gauss_points(n, n, L, L)
    shift = lambda pts: [(x - 5.0, y - 5.0) for (x, y) in pts]
    Wx = _point_state(lambda x, y: isotropic_vortex_state(x, y, gamma, eps), shift(wxp))
    Wy = _point_state(lambda x, y: isotropic_vortex_state(x, y, gamma, eps), shift(wyp))
    bc = [(BC_PERIODIC, 0.0, 0.0, 1.0)] * 4
    return Problem(f"isotropic_vortex_{n}", n, n, L, L, gamma, 0.0, 1.0, bc,
                   np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy),
                   meta={"eps": eps, "period": 10.0})


def sod(nx: int, gamma: float = 1.4) -> Problem:
    """Sod's shock tube on [0, 1] (diaphragm at x = 0.5) as an nx-by-1 grid, dy = dx."""
    return shock_tube(nx, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), gamma, name=f"sod_{nx}")


def shock_tube(nx: int, left, right, gamma: float = 1.4, name: str | None = None) -> Problem:
    """A Riemann problem on [0, 1] with primitive states left = (rho, u, p) for x < 0.5 and
    right for x > 0.5, as an nx-by-1 grid (dy = dx), periodic in y, outflow ends."""
    Lx = 1.0
    dx = Lx / nx
    left = _cons(left[0], left[1], 0.0, left[2], gamma)
    right = _cons(right[0], right[1], 0.0, right[2], gamma)
    xl = np.arange(nx) * dx
    fr = np.clip((xl + dx - 0.5) / dx, 0.0, 1.0)  # fraction of the cell right of x = 0.5
    U = (left.reshape(4, 1) * (1 - fr) + right.reshape(4, 1) * fr)[:, None, :]

    def pt(x, y):
        x = np.asarray(x, dtype=np.float64)
        s = np.where(x > 0.5, 1.0, np.where(x < 0.5, 0.0, 0.5))
        return left.reshape(4, *([1] * x.ndim)) * (1 - s) + right.reshape(4, *([1] * x.ndim)) * s

    _, _, wxp, wyp = _gauss_points(nx, 1, Lx, dx)
    Wx = _point_state(pt, wxp)
    Wy = _point_state(pt, wyp)
    bc = [(BC_OUTFLOW, 0.0, 0.0, 1.0), (BC_OUTFLOW, 0.0, 0.0, 1.0), (BC_PERIODIC, 0.0, 0.0, 1.0),
          (BC_PERIODIC, 0.0, 0.0, 1.0)]
    return Problem(name or f"shock_tube_{nx}", nx, 1, Lx, dx, gamma, 0.0, 1.0, bc,
                   np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy))


def _piecewise_x(nx, ny, Lx, Ly, breaks, states, gamma):
    """Cell averages and Gauss-point values of primitive states constant on x-intervals:
    states[k] = (rho, u, p) on [breaks[k], breaks[k + 1]); cells cut by a break take the
    length-weighted mix, points exactly on a break the mean of the two sides."""
    dx = Lx / nx
    cons = [_cons(r, u, 0.0, p, gamma) for (r, u, p) in states]
    xl = np.arange(nx) * dx
    avg = np.zeros((4, nx))
    for k, c in enumerate(cons):
        lo, hi = breaks[k], breaks[k + 1]
        xr = (np.arange(nx) + 1) * dx
        part = np.clip((np.minimum(xr, hi) - np.maximum(xl, lo)) / dx, 0.0, 1.0)
        frac = np.where((xl >= lo) & (xr <= hi), 1.0, np.where((xr <= lo) | (xl >= hi), 0.0, part))
        avg += c.reshape(4, 1) * frac
    U = np.ascontiguousarray(np.broadcast_to(avg[:, None, :], (4, ny, nx)).copy())

    def pt(x, y):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros((4,) + x.shape)
        for k, c in enumerate(cons):
            lo, hi = breaks[k], breaks[k + 1]
            w = np.where((x > lo) & (x < hi), 1.0, 0.0)
            w = w + 0.5 * (np.isclose(x, lo) & (k > 0)) + 0.5 * (np.isclose(x, hi) & (k < len(cons) - 1))
            w = w + 1.0 * (np.isclose(x, lo) & (k == 0)) + 1.0 * (np.isclose(x, hi) & (k == len(cons) - 1))
            out += c.reshape(4, *([1] * x.ndim)) * w
        return out

    _, _, wxp, wyp = _gauss_points(nx, ny, Lx, Ly)
    return U, np.ascontiguousarray(_point_state(pt, wxp)), np.ascontiguousarray(_point_state(pt, wyp))


def blast_wave(nx: int = 400, gamma: float = 1.4) -> Problem:
    """The Woodward-Colella blast wave of Section 5 (1D tests): [0, 100], (rho, u, p) =
    (1, 0, 1000) for x < 10, (1, 0, 0.01) on [10, 90), (1, 0, 100) beyond; reflecting ends
    (slip walls), as an nx-by-1 grid (dy = dx, periodic in y).  The paper runs 400 cells to
    t = 3.8."""
    Lx = 100.0
    dx = Lx / nx
    U, Wx, Wy = _piecewise_x(nx, 1, Lx, dx, [0.0, 10.0, 90.0, 100.0],
                             [(1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), (1.0, 0.0, 100.0)], gamma)
    wall = (BC_SLIPWALL, 0.0, 0.0, 1.0)
    bc = [wall, wall, (BC_PERIODIC, 0.0, 0.0, 1.0), (BC_PERIODIC, 0.0, 0.0, 1.0)]
    return Problem(f"blast_wave_{nx}", nx, 1, Lx, dx, gamma, 0.0, 1.0, bc, U, Wx, Wy,
                   meta={"t_end": 3.8})


def viscous_shock_tube(nx: int = 300, Re: float = 200.0, gamma: float = 1.4, Pr: float = 0.73) -> Problem:
    """The viscous shock tube of Section 5: gas at rest in [0, 1] x [0, 0.5], (rho, u, p) =
    (120, 0, 120/gamma) for x < 0.5 and (1.2, 0, 1.2/gamma) beyond; adiabatic no-slip walls
    at x = 0, x = 1 and y = 0, symmetry (slip wall) at y = 0.5; Pr = 0.73, mu = 1/Re (the
    reading of the Reynolds number: unit reference density, velocity and length); nx by
    nx / 2 cells (the paper: 300 x 150 at Re = 200), to t = 1."""
    ny = nx // 2
    Lx, Ly = 1.0, 0.5
    U, Wx, Wy = _piecewise_x(nx, ny, Lx, Ly, [0.0, 0.5, 1.0],
                             [(120.0, 0.0, 120.0 / gamma), (1.2, 0.0, 1.2 / gamma)], gamma)
    wall = (BC_NOSLIP_ADIABATIC, 0.0, 0.0, 1.0)
    bc = [wall, wall, wall, (BC_SLIPWALL, 0.0, 0.0, 1.0)]
    return Problem(f"viscous_shock_tube_{nx}x{ny}", nx, ny, Lx, Ly, gamma, 1.0 / Re, Pr, bc, U, Wx, Wy,
                   meta={"Re": Re, "t_end": 1.0})


BATCH_SIZES = [32 * k for k in range(1, 13)]


def batch_specs(n_grids: int = 512, seed: int = 5):
    """Per grid: (nx, ny, kind, gamma, mu, draws) with kind 'wave' for even g, 'riemann' for odd."""
    rng = SplitMix64(seed)
    specs = []
    for g in range(n_grids):
        nx = BATCH_SIZES[min(int(rng.uniform() * 12), 11)]
        ny = BATCH_SIZES[min(int(rng.uniform() * 12), 11)]
        gamma = 1.4 if rng.uniform() < 0.5 else 5.0 / 3.0
        mu = 10.0 ** (-5.0 + 2.0 * rng.uniform())
        if g % 2 == 0:
            specs.append((nx, ny, "wave", gamma, mu, rng.uniform()))
        else:
            specs.append((nx, ny, "riemann", gamma, mu, riemann_draw(rng)))
    return specs


def batch_problem(spec) -> Problem:
    nx, ny, kind, gamma, mu, draw = spec
    if kind == "wave":
        p = smooth_wave_2d(nx, ny=ny, gamma=gamma)
        # replace the phase by the batch draw
        return _rephase(p, draw, gamma, mu)
    return riemann_2d(nx, ny, gamma=gamma, mu=mu, Pr=0.72, quadrants=draw)


def _rephase(p: Problem, phi: float, gamma: float, mu: float) -> Problem:
    nx, ny, Lx, Ly = p.nx, p.ny, p.Lx, p.Ly
    dx, dy = Lx / nx, Ly / ny
    xc, yc, wxp, wyp = _gauss_points(nx, ny, Lx, Ly)
    X, Y = np.meshgrid(xc, yc)
    rho_bar = 1.0 + 0.2 * np.sin(np.pi * (X + Y) + phi) * sinc(np.pi * dx / 2) * sinc(np.pi * dy / 2)
    U = np.stack([rho_bar, rho_bar, rho_bar, 1.0 / (gamma - 1.0) + rho_bar])

    def pt(x, y):
        r = 1.0 + 0.2 * np.sin(np.pi * (x + y) + phi)
        return _cons(r, 1.0, 1.0, 1.0, gamma)

    return Problem(f"wave_{nx}x{ny}", nx, ny, Lx, Ly, gamma, mu, 0.72, p.bc, np.ascontiguousarray(U),
                   np.ascontiguousarray(_point_state(pt, wxp)), np.ascontiguousarray(_point_state(pt, wyp)),
                   meta={"phi": phi})
