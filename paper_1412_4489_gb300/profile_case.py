"""Runs a few time steps of one seeded workload through the library, one step per
``gks_step`` call, so that a profiler sees each step's kernels in launch order
(begin, ghost, recon, flux_x, flux_y, update passes 1-3, end).

    python -m paper_1412_4489_gb300.profile_case --workload smooth --size 2048 --precision fp32 --steps 3

Workloads: ``smooth`` (2D Euler density wave, periodic, collision time tau_eps = 0),
``riemann`` (Navier-Stokes four-quadrant data, mu = 1e-4, outflow) and ``cavity``
(lid-driven cavity, isothermal no-slip walls); ``batch`` takes ``--size`` seeded grids of the
batched form (sizes 32..384, smooth waves and Navier-Stokes Riemann data) and advances them one
persistent launch per step.
"""
from __future__ import annotations

import argparse

from . import gks, workloads as wl


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=("smooth", "riemann", "cavity", "batch"), default="smooth")
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--precision", choices=("fp32", "fp64"), default="fp32")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--cfl", type=float, default=0.5)
    a = ap.parse_args(argv)
    prec = gks.GKS_FP32_BULK if a.precision == "fp32" else gks.GKS_FP64
    if a.workload == "batch":
        probs = [wl.batch_problem(sp) for sp in wl.batch_specs(a.size, seed=5)]
        b = gks.Batch(probs, prec)
        for _ in range(a.steps):
            b.step(1, a.cfl)
        lo, hi = b.sync()
        b.close()
        cells = sum(p.nx * p.ny for p in probs)
        print(f"batch of {a.size} grids ({cells} cells) {a.precision}: {lo}..{hi} steps")
        return
    if a.workload == "smooth":
        p, te = wl.smooth_wave_2d(a.size, seed=2), 0.0
    elif a.workload == "riemann":
        p, te = wl.riemann_2d(a.size, seed=3, mu=1e-4, Pr=0.72), 0.05
    else:
        p, te = wl.cavity_2d(a.size), 0.05
    s = gks.Solver(p, prec, tau_eps=te)
    for _ in range(a.steps):
        s.step(a.cfl)
    t, n = s.sync()
    s.close()
    print(f"{a.workload} {a.size}^2 {a.precision}: {n} steps, t = {t:.6g}")


if __name__ == "__main__":
    main()
