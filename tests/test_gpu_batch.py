"""GPU checks of the batched form: one persistent launch advancing grids of uneven sizes,
kinds, gamma and viscosity must give, grid by grid, the states of the single-grid path
(which the other GPU tests pin to the oracle), and the oracle itself on a subset."""
import numpy as np
import pytest

import oracle
from paper_1412_4489_gb300 import gks, workloads as wl

pytestmark = pytest.mark.gpu


def _mixed_grids():
    ps = [wl.smooth_wave_2d(37, ny=29, seed=2),
          wl.riemann_2d(45, 38, seed=3, mu=1e-3, Pr=0.72),
          wl.riemann_2d(20, 66, seed=4, mu=0.0, Pr=1.0, gamma=5.0 / 3.0),
          wl.cavity_2d(24),
          wl.smooth_wave_2d(64, ny=33, seed=7, gamma=5.0 / 3.0)]
    ps[0].mu, ps[0].Pr = 2e-4, 0.72
    return ps


@pytest.mark.parametrize("prec", [gks.GKS_FP64, gks.GKS_FP32_BULK])
def test_batch_matches_single_grid_path(prec):
    ps = _mixed_grids()
    b = gks.Batch(ps, prec)
    b.step(12, 0.5)
    lo, hi = b.sync()
    assert lo == hi == 12
    # FP64: the same arithmetic to roundoff.  FP32: the batched and single-grid kernels
    # are compiled separately, and roundoff-level differences in their code generation
    # flip limiter and stencil choices at the discontinuities of the Riemann grid, each
    # flip moving a few cells by up to ~1e-3 of the state; so the comparison is the
    # relative L1 norm within the FP32 error budget against FP64 (1e-5; the two agree
    # to ~1e-6), with a loose Linf (3e-3) that only catches gross errors
    tol = 1e-12 if prec == gks.GKS_FP64 else 3e-3
    for g, p in enumerate(ps):
        s = gks.Solver(p, prec)
        for _ in range(12):
            s.step(0.5)
        U, Wx, Wy, t = s.state()
        s.close()
        Ub, Wxb, Wyb, tb, nb = b.state(g)
        assert nb == 12
        assert tb == pytest.approx(t, rel=1e-12 if prec == gks.GKS_FP64 else 2e-4)
        for got, want in ((Ub, U), (Wxb, Wx), (Wyb, Wy)):
            if prec == gks.GKS_FP32_BULK:
                assert np.sum(np.abs(got - want)) <= 1e-5 * np.sum(np.abs(want))
            assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    b.close()


def test_batch_against_the_oracle():
    ps = [wl.riemann_2d(30, 22, seed=11, mu=5e-4, Pr=0.72), wl.smooth_wave_2d(26, ny=34, seed=5)]
    b = gks.Batch(ps, gks.GKS_FP64)
    b.step(15, 0.5)
    b.sync()
    for g, p in enumerate(ps):
        P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr)
        st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
        bc = oracle.bcs([q[0] for q in p.bc], [q[1:] for q in p.bc])
        for _ in range(15):
            assert oracle.step2d(P, st, bc, 0.5)[0] == 0
        U, _, _, t, _ = b.state(g)
        assert t == pytest.approx(st.t, rel=1e-12)
        assert np.max(np.abs(U - st.U)) <= 1e-10 * np.max(np.abs(st.U))
    b.close()


def test_autotune_keeps_the_state():
    ps = _mixed_grids()[:3]
    b = gks.Batch(ps, gks.GKS_FP32_BULK)
    before = [b.state(g) for g in range(len(ps))]
    (wx, wy), k, ms = gks.gks_batch_autotune(b.b, 0.5, 1)
    assert wx in (4, 8, 16, 32) and wy in (16, 32, 64, 128) and k >= 1 and ms > 0
    for g in range(len(ps)):
        after = b.state(g)
        for x, y in zip(before[g][:3], after[:3]):
            assert np.array_equal(x, y)
        assert after[4] == before[g][4]
    b.step(3, 0.5)
    assert b.sync() == (3, 3)
    b.close()


def test_barrier_wait_times_out_instead_of_hanging():
    """A test hook makes block 0 skip its barrier arrivals; every other wait runs out after
    0.2 s and the call reports GKS_ETIMEOUT.  The context stays usable."""
    ps = _mixed_grids()[:2]
    b = gks.Batch(ps, gks.GKS_FP32_BULK)
    gks.gks_batch_set_wait_limit(b.b, 0.2, 0)
    b.step(2, 0.5)
    with pytest.raises(gks.GKSError) as e:
        b.sync()
    assert e.value.status == gks.GKS_ETIMEOUT
    b.close()
    c = gks.Batch(ps, gks.GKS_FP32_BULK)
    c.step(2, 0.5)
    assert c.sync() == (2, 2)
    c.close()


def _bench_subset(n):
    """The first n grids of the benchmark's 512-grid batch (sizes 32..384, both kinds, both
    gammas, mu ~ logU[1e-5, 1e-3])."""
    return [wl.batch_problem(sp) for sp in wl.batch_specs(512, seed=5)[:n]]


def test_benchmark_batch_subset_fp64_against_the_oracle():
    """16 grids of the benchmark batch in one persistent launch, FP64, against the oracle run
    grid by grid (the oracle on the host cores): rel-Linf 1e-10 on the smooth waves, L1 1e-8 on
    the four-quadrant data."""
    ps = _bench_subset(16)
    b = gks.Batch(ps, gks.GKS_FP64)
    n = 3
    b.step(n, 0.5)
    b.sync()
    for g, p in enumerate(ps):
        P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr)
        st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
        bc = oracle.bcs([q[0] for q in p.bc], [q[1:] for q in p.bc])
        for _ in range(n):
            assert oracle.step2d(P, st, bc, 0.5)[0] == 0
        U, _, _, t, _ = b.state(g)
        assert t == pytest.approx(st.t, rel=1e-12)
        if p.bc[0][0] == wl.BC_PERIODIC:
            assert np.max(np.abs(U - st.U)) <= 1e-10 * np.max(np.abs(st.U)), g
        else:
            assert np.sum(np.abs(U[0] - st.U[0])) <= 1e-8 * np.sum(np.abs(st.U[0])), g
    b.close()


def test_benchmark_batch_fp32_bulk_l1_per_grid():
    """The FP32-bulk batch against the FP64 batch, grid by grid: relative L1 of density within
    1e-5 after the steps the benchmark times."""
    ps = _bench_subset(64)
    a, c = gks.Batch(ps, gks.GKS_FP64), gks.Batch(ps, gks.GKS_FP32_BULK)
    for b in (a, c):
        b.step(6, 0.5)
        b.sync()
    worst = 0.0
    for g in range(len(ps)):
        U64, U32 = a.state(g)[0], c.state(g)[0]
        worst = max(worst, np.sum(np.abs(U32[0] - U64[0])) / np.sum(np.abs(U64[0])))
    a.close()
    c.close()
    assert worst <= 1e-5, worst
