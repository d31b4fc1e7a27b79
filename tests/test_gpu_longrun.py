"""Long-run parity at full size: the GPU FP64 path against stored oracle results at sampled
cells, written by tests/golden/make_longrun.py (which runs only the oracle): the 512^2
lid-driven cavity after 1000 steps and the 1024^2 Navier-Stokes four-quadrant data after 100
steps (the predictability horizon of that workload: past it a 1e-12 perturbation of the start
grows to 1e-2, see test_gpu_fullsize.py)."""
import os

import numpy as np
import pytest

from paper_1412_4489_gb300 import gks, workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated (python tests/golden/make_longrun.py)")
    meta, rows = {}, []
    for line in open(path):
        if line.startswith("# nx"):
            f = line[1:].split()
            meta = {f[k]: f[k + 1] for k in range(0, len(f) - 1, 2)}
        elif not line.startswith("#") and line.strip():
            rows.append([float(x) for x in line.split()])
    rows = np.array(rows)
    return meta, rows[:, 0].astype(int), rows[:, 1].astype(int), rows[:, 2:]


@pytest.mark.parametrize("case", ["cavity_512_1000", "riemann_ns_1024_100"])
def test_fp64_long_run_matches_the_oracle(case):
    meta, jj, ii, want = _load(f"longrun_{case}.txt")
    if case.startswith("cavity"):
        # smooth: rel-Linf 1e-10 per 100 steps, roundoff differences (FMA contraction, closed-form
        # against eliminated 4x4 solves) accumulating over the 1000 steps
        p, n, tol = wl.cavity_2d(512), 1000, 1e-9
    else:
        p, n, tol = wl.riemann_2d(1024, seed=3, mu=1e-4, Pr=0.72), 100, 1e-8  # discontinuous
    assert int(meta["nx"]) == p.nx and int(meta["ny"]) == p.ny
    s = gks.Solver(p, gks.GKS_FP64, tau_eps=0.05, weno_C=1.0)  # the references' constant
    s.advance(n, 0.5)
    U, _, _, t = s.state()
    s.close()
    assert t == pytest.approx(float(meta["t"]), rel=1e-12)
    got = U[:, jj, ii].T
    scale = np.abs(U).reshape(4, -1).max(axis=1)
    err = np.max(np.abs(got - want) / scale)
    assert err <= tol, err
