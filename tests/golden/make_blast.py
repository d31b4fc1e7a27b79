"""Writes blast_wave_400_t3.8.txt, the FP64 oracle's cell averages of the Woodward-Colella
blast wave (Section 5, 1D tests: 400 cells on [0, 100], reflecting ends, gamma 1.4) after
150 steps and at t = 3.8, with CFL 0.5, tau_eps 0.05 and the last step clipped to reach
t = 3.8 exactly.  The header also records the oracle's own sensitivity at t = 3.8: the
relative L1 distance to this run of (a) the same run started from cell averages perturbed
by 1e-14 (seeded normal noise) and (b) one started from face point values rounded to FP32.
Only the oracle runs here (about a minute and a half on one core):

    python tests/golden/make_blast.py
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

CFL, T_END, CHECK = 0.5, 3.8, 150


def run(p, U, Wx, Wy):
    """(state after CHECK steps, state at T_END, steps)"""
    P = oracle.params(gamma=p.gamma, tau_eps=0.05)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, U, Wx, Wy)
    bc = oracle.bcs([b[0] for b in p.bc])
    n, early = 0, None
    while st.t < T_END:
        rc, _ = oracle.step2d(P, st, bc, CFL, dt_max=T_END - st.t)
        if rc != 0:
            raise RuntimeError(f"blast wave: oracle step {n} failed ({rc})")
        n += 1
        if n == CHECK:
            early = st.U[:, 0, :].copy()
    return early, st.U[:, 0, :].copy(), n


def l1(a, b):
    return np.abs(a - b).sum(axis=1) / np.abs(b).sum(axis=1)


def main() -> None:
    p = wl.blast_wave(400)
    t0 = time.time()
    early, final, n = run(p, p.U, p.Wx, p.Wy)
    noise = np.random.default_rng(7).standard_normal(p.U.shape)
    _, fa, _ = run(p, p.U * (1.0 + 1e-14 * noise), p.Wx, p.Wy)
    _, fb, _ = run(p, p.U, p.Wx.astype(np.float32).astype(np.float64), p.Wy.astype(np.float32).astype(np.float64))
    ca, cb = l1(fa, final), l1(fb, final)
    with open(os.path.join(HERE, "blast_wave_400_t3.8.txt"), "w") as f:
        f.write(f"# Woodward-Colella blast wave, 400 cells: FP64 oracle after {CHECK} steps and at t = {T_END} "
                f"({n} steps; CFL {CFL}, tau_eps 0.05), written by tests/golden/make_blast.py from oracle/ only\n")
        f.write(f"# nx {p.nx} steps {n} check {CHECK} seconds {time.time() - t0:.0f}\n")
        f.write("# sensitivity_u1e-14 " + " ".join(repr(float(x)) for x in ca) + "\n")
        f.write("# sensitivity_w_fp32 " + " ".join(repr(float(x)) for x in cb) + "\n")
        f.write("# columns: stage i rho rhoU rhoV rhoE (stage 0: after the check steps, 1: at t_end)\n")
        for stage, U in ((0, early), (1, final)):
            for i in range(p.nx):
                f.write(f"{stage} {i} " + " ".join(repr(float(x)) for x in U[:, i]) + "\n")


if __name__ == "__main__":
    main()
