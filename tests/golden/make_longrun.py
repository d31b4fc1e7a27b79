"""Writes the long-run oracle references that tests/test_gpu_longrun.py compares the GPU FP64
path against, as values at sampled cells (the whole fields would be megabytes):

  longrun_cavity_512_1000.txt       lid-driven cavity 512^2, 1000 steps
  longrun_riemann_ns_1024_100.txt   Navier-Stokes four-quadrant data 1024^2, 100 steps

Both with CFL 0.5 and tau_eps 0.05, from the seeded workload generators.  Only the FP64
oracle runs here (about an hour on 8 cores for both):

    python tests/golden/make_longrun.py [cavity|riemann ...]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1412_4489_gb300 import workloads as wl  # noqa: E402

CFL = 0.5
WENO_C = 1.0  # the constant of I(U1) these references were generated with (a parity check: any value)


def sample_cells(nx: int, ny: int, seed: int, lines: bool) -> list[tuple[int, int]]:
    """Seeded random cells, the boundary rows and columns, the corners and, for the
    four-quadrant data, cells along the two initial discontinuity lines."""
    rng = np.random.default_rng(seed)
    cells = {(int(j), int(i)) for j, i in zip(rng.integers(0, ny, 400), rng.integers(0, nx, 400))}
    for k in range(0, nx, max(1, nx // 32)):
        cells |= {(0, k), (ny - 1, k)}
    for k in range(0, ny, max(1, ny // 32)):
        cells |= {(k, 0), (k, nx - 1)}
    cells |= {(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)}
    if lines:
        for k in range(0, nx, 8):
            cells |= {(ny // 2 - 1, k), (ny // 2, k)}
        for k in range(0, ny, 8):
            cells |= {(k, nx // 2 - 1), (k, nx // 2)}
    return sorted(cells)


def run(name: str, p, bc, nsteps: int, seed: int, lines: bool, out: str) -> None:
    P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr, tau_eps=0.05, weno_C=WENO_C)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
    t0 = time.time()
    for k in range(nsteps):
        rc, _ = oracle.step2d(P, st, bc, CFL)
        if rc != 0:
            raise RuntimeError(f"{name}: oracle step {k} failed ({rc})")
    cells = sample_cells(p.nx, p.ny, seed, lines)
    with open(out, "w") as f:
        f.write(f"# {name}: FP64 oracle after {nsteps} steps (CFL {CFL}, tau_eps 0.05, weno_C {WENO_C}), written by "
                f"tests/golden/make_longrun.py from oracle/ only\n")
        f.write(f"# nx {p.nx} ny {p.ny} t {st.t!r} threads {oracle.num_threads()} seconds {time.time() - t0:.0f}\n")
        f.write("# columns: j i rho rhoU rhoV rhoE\n")
        for j, i in cells:
            f.write(f"{j} {i} " + " ".join(repr(float(x)) for x in st.U[:, j, i]) + "\n")


def main(which: list[str]) -> None:
    if "cavity" in which:
        p = wl.cavity_2d(512)
        bc = oracle.bcs([b[0] for b in p.bc], [b[1:] for b in p.bc])
        run("lid-driven cavity 512^2 (Re 1000, lid Mach 0.15)", p, bc, 1000, 21, False,
            os.path.join(HERE, "longrun_cavity_512_1000.txt"))
    if "riemann" in which:
        p = wl.riemann_2d(1024, seed=3, mu=1e-4, Pr=0.72)
        bc = oracle.bcs([b[0] for b in p.bc])
        run("Navier-Stokes four-quadrant data 1024^2 (seed 3, mu 1e-4, Pr 0.72)", p, bc, 100, 22, True,
            os.path.join(HERE, "longrun_riemann_ns_1024_100.txt"))


if __name__ == "__main__":
    main(sys.argv[1:] or ["cavity", "riemann"])
