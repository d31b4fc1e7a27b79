"""Parity at the workloads' full sizes: one GPU step against the oracle on sampled cells
(the oracle evaluates only the faces of those cells), and properties that hold at any size.
Also FP32-bulk against the FP64 oracle in L1 at moderate sizes."""
import numpy as np
import pytest

import oracle
from paper_1412_4489_gb300 import gks, workloads as wl

pytestmark = pytest.mark.gpu


def _sample_cells(p, n, seed):
    rng = np.random.default_rng(seed)
    cells = {(int(j), int(i)) for j, i in zip(rng.integers(0, p.ny, n), rng.integers(0, p.nx, n))}
    # boundary rows / columns and the corners
    for k in range(0, p.nx, max(1, p.nx // 16)):
        cells |= {(0, k), (p.ny - 1, k)}
    for k in range(0, p.ny, max(1, p.ny // 16)):
        cells |= {(k, 0), (k, p.nx - 1)}
    cells |= {(0, 0), (0, p.nx - 1), (p.ny - 1, 0), (p.ny - 1, p.nx - 1)}
    return sorted(cells)


def _oracle_one_step_at(p, cells, tau_eps=0.05):
    P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr, tau_eps=tau_eps)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
    bc = oracle.bcs([b[0] for b in p.bc], [b[1:] for b in p.bc])
    dt = oracle.dt2d(P, st, 0.5)
    faces = []
    for j, i in cells:
        faces += [(0, i, j), (0, i + 1, j), (1, i, j), (1, i, j + 1)]
    F, W = oracle.flux2d_faces(P, st, bc, dt, faces)
    dx, dy = p.Lx / p.nx, p.Ly / p.ny
    Un = np.array([p.U[:, j, i] + (F[4 * k] - F[4 * k + 1]) / dx + (F[4 * k + 2] - F[4 * k + 3]) / dy
                   for k, (j, i) in enumerate(cells)])
    return dt, Un, F, W, faces


@pytest.mark.parametrize("case", ["riemann_ns_1024", "cavity_512", "smooth_512"])
def test_one_step_sampled_fp64(case):
    if case == "riemann_ns_1024":
        p, te = wl.riemann_2d(1024, seed=3, mu=1e-4, Pr=0.72), 0.05
    elif case == "cavity_512":
        p, te = wl.cavity_2d(512), 0.05
    else:
        p, te = wl.smooth_wave_2d(512, seed=2), 0.0
    cells = _sample_cells(p, 300, seed=1)
    dt_o, Un_o, F, W, faces = _oracle_one_step_at(p, cells, te)
    s = gks.Solver(p, gks.GKS_FP64, tau_eps=te)
    dt_g = s.step(0.5)
    U, Wx, Wy, _ = s.state()
    s.close()
    assert dt_g == pytest.approx(dt_o, rel=1e-13)
    got = np.array([U[:, j, i] for j, i in cells])
    scale = np.abs(p.U).max()  # one scale: momenta can vanish (cavity at rest)
    assert np.max(np.abs(got - Un_o) / scale) < 1e-12
    for k, (ax, i, j) in enumerate(faces):
        Wg = Wx[:, :, j, i].T if ax == 0 else Wy[:, :, j, i].T
        assert np.max(np.abs(Wg - W[k]) / scale) < 1e-11


def test_one_step_sampled_fp32_bulk_bench_configuration():
    """The configuration bench.py times: the 512^2 smooth wave in FP32-bulk."""
    p = wl.smooth_wave_2d(512, seed=2)
    cells = _sample_cells(p, 300, seed=2)
    dt_o, Un_o, _, _, _ = _oracle_one_step_at(p, cells, 0.0)
    s = gks.Solver(p, gks.GKS_FP32_BULK, tau_eps=0.0)
    dt_g = s.step(0.5)
    U, _, _, _ = s.state()
    s.close()
    assert dt_g == pytest.approx(dt_o, rel=1e-6)
    got = np.array([U[:, j, i] for j, i in cells])
    inc = np.abs(Un_o - np.array([p.U[:, j, i] for j, i in cells])).max(axis=0)
    # the FP32 face evolution errs by ~1e-6 of the per-step change, the FP64 accumulation adds nothing
    assert np.all(np.max(np.abs(got - Un_o), axis=0) <= 1e-5 * inc + 1e-12)


@pytest.mark.parametrize("prec", [gks.GKS_FP64, gks.GKS_FP32_BULK])
def test_conservation_at_full_size(prec):
    """Periodic 512^2: the face fluxes telescope, so total mass, momentum and energy are
    conserved to FP64 roundoff in both precisions."""
    p = wl.smooth_wave_2d(512, seed=2)
    s = gks.Solver(p, prec, tau_eps=0.0)
    s.advance(20, 0.5)
    U, _, _, _ = s.state()
    s.close()
    tot0, tot = p.U.sum(axis=(1, 2)), U.sum(axis=(1, 2))
    np.testing.assert_allclose(tot, tot0, rtol=1e-12)


@pytest.mark.parametrize("case", ["smooth", "riemann_ns"])
def test_fp32_bulk_against_fp64_oracle_l1(case):
    """The FP32-bulk form's density error against the FP64 oracle, relative L1 <= 1e-5."""
    if case == "smooth":
        p, n, te = wl.smooth_wave_2d(64, ny=48, seed=2), 100, 0.0
    else:
        p, n, te = wl.riemann_2d(48, 40, seed=3, mu=1e-4, Pr=0.72), 50, 0.05
    P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr, tau_eps=te)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
    bc = oracle.bcs([b[0] for b in p.bc])
    s = gks.Solver(p, gks.GKS_FP32_BULK, tau_eps=te)
    for _ in range(n):
        s.step(0.5)
        assert oracle.step2d(P, st, bc, 0.5)[0] == 0
    U, _, _, _ = s.state()
    s.close()
    l1 = np.sum(np.abs(U[0] - st.U[0])) / np.sum(np.abs(st.U[0]))
    assert l1 <= 1e-5, l1
