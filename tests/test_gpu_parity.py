"""GPU parity: the CUDA path through the C ABI against the oracle, element by element.

Grids are sized to span several thread blocks with ragged tails; every boundary kind and
both the Euler and Navier-Stokes models are covered.  FP64 tolerance: the paper fixes no
precision; both sides compute in FP64 with different operation orders, so single-kernel
outputs agree to ~1e-13 and 100-step states to rel-Linf 1e-10 on smooth data and L1 1e-8
on discontinuous data (limiter branches can flip at roundoff-level ties).
"""
import numpy as np
import pytest

import oracle
from paper_1412_4489_gb300 import gks, workloads as wl

pytestmark = pytest.mark.gpu

PER = [wl.BC_PERIODIC] * 4


def _oracle_params(p, **kw):
    return oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr, **kw)


def _oracle_bc(p):
    return oracle.bcs([b[0] for b in p.bc], [b[1:] for b in p.bc])


def _perturbed(nx, ny, seed, bc=PER, mu=0.0, Pr=1.0, amp=0.05):
    p = wl.smooth_wave_2d(nx, ny=ny, seed=seed)
    rng = np.random.default_rng(seed)
    sc = np.array([1, 1, 1, 0.2])
    p.U = np.ascontiguousarray(p.U * (1 + amp * rng.uniform(-1, 1, p.U.shape) * sc[:, None, None]))
    p.Wx = np.ascontiguousarray(p.Wx * (1 + amp * rng.uniform(-1, 1, p.Wx.shape) * sc[:, None, None, None]))
    p.Wy = np.ascontiguousarray(p.Wy * (1 + amp * rng.uniform(-1, 1, p.Wy.shape) * sc[:, None, None, None]))
    if bc[0] == wl.BC_PERIODIC:
        p.Wx[..., -1] = p.Wx[..., 0]
    if bc[2] == wl.BC_PERIODIC:
        p.Wy[:, :, -1, :] = p.Wy[:, :, 0, :]
    p.bc = [b if isinstance(b, tuple) else (b, 0.0, 0.0, 1.0) for b in bc]
    p.mu, p.Pr = mu, Pr
    return p


def _state(p):
    return oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)


BCSETS = {
    "periodic": PER,
    "outflow": [wl.BC_OUTFLOW] * 4,
    "slip": [wl.BC_SLIPWALL] * 4,
    "noslip": [(wl.BC_NOSLIP_ISOTHERMAL, 0.0, 0.0, 0.9), (wl.BC_NOSLIP_ISOTHERMAL, 0.0, 0.1, 1.1),
               (wl.BC_NOSLIP_ISOTHERMAL, -0.1, 0.0, 1.0), (wl.BC_NOSLIP_ISOTHERMAL, 0.15, 0.0, 1.0)],
    "mixed": [wl.BC_PERIODIC, wl.BC_PERIODIC, wl.BC_SLIPWALL, wl.BC_OUTFLOW],
    "adiabatic": [(wl.BC_NOSLIP_ADIABATIC, 0.0, 0.0, 1.0), (wl.BC_NOSLIP_ADIABATIC, 0.0, -0.1, 1.0),
                  (wl.BC_NOSLIP_ADIABATIC, 0.12, 0.0, 1.0), (wl.BC_NOSLIP_ISOTHERMAL, 0.0, 0.0, 1.0)],
}


@pytest.mark.parametrize("bcname", list(BCSETS))
def test_reconstruction_parity(bcname):
    p = _perturbed(37, 29, seed=1, bc=BCSETS[bcname])
    s = gks.Solver(p)
    got = gks.gks_debug_recon(s.h, p.nx, p.ny)
    s.close()
    want = oracle.recon2d(_oracle_params(p), _state(p), _oracle_bc(p))
    scale = np.abs(want).reshape(4, 6, -1).max(axis=2)[:, :, None, None] + 1e-300
    np.testing.assert_allclose(got / scale, want / scale, rtol=0, atol=1e-12)


@pytest.mark.parametrize("bcname", list(BCSETS))
@pytest.mark.parametrize("mu,Pr", [(0.0, 1.0), (2e-3, 0.72)])
def test_face_flux_parity(bcname, mu, Pr):
    p = _perturbed(35, 26, seed=2, bc=BCSETS[bcname], mu=mu, Pr=Pr)
    dt = 0.4 * oracle.dt2d(_oracle_params(p), _state(p), 1.0)
    s = gks.Solver(p)
    Fx, Fy, Wx, Wy = gks.gks_debug_flux(s.h, p.nx, p.ny, dt)
    s.close()
    oFx, oFy, oWx, oWy = oracle.flux2d(_oracle_params(p), _state(p), _oracle_bc(p), dt)
    for got, want in ((Fx, oFx), (Fy, oFy), (Wx, oWx), (Wy, oWy)):
        scale = np.abs(want).reshape(want.shape[0], -1).max(axis=1).reshape(-1, *([1] * (want.ndim - 1)))
        np.testing.assert_allclose(got / scale, want / scale, rtol=0, atol=1e-12)


def _run_both(p, nsteps, cfl=0.5, P=None, **opts):
    P = P or _oracle_params(p)
    s = gks.Solver(p, gks.GKS_FP64, **opts)
    st = _state(p)
    bc = _oracle_bc(p)
    for _ in range(nsteps):
        dg = s.step(cfl)
        rc, do = oracle.step2d(P, st, bc, cfl)
        assert rc == 0
        assert dg == pytest.approx(do, rel=1e-12)
    U, Wx, Wy, t = s.state()
    s.close()
    return (U, Wx, Wy), (st.U, st.Wx, st.Wy)


def _rel_linf(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_smooth_wave_100_steps():
    p = wl.smooth_wave_2d(48, ny=40, seed=2)
    g, o = _run_both(p, 100, P=oracle.params(gamma=1.4, tau_eps=0.0), tau_eps=0.0)
    for a, b in zip(g, o):
        assert _rel_linf(a, b) < 1e-10


@pytest.mark.parametrize("bcname", ["periodic", "noslip", "adiabatic"])
def test_rows_of_whole_warps_of_x_faces(bcname):
    """nx a multiple of 32: the last x-face of every row (a periodic seam or a wall face) is
    evaluated by the extra column of blocks that takes it 128 rows at a time.  Every face and
    cell against the oracle over 8 steps (ny = 200 spans two of those blocks)."""
    p = _perturbed(64, 200, seed=11, bc=BCSETS[bcname], mu=1e-3, Pr=0.72)
    g, o = _run_both(p, 8)
    for a, b in zip(g, o):
        assert _rel_linf(a, b) < 1e-10


_TINY = [((1, 1), "periodic"), ((1, 7), "periodic"), ((7, 1), "periodic"), ((2, 2), "periodic"), ((3, 5), "periodic"),
         ((2, 2), "outflow"), ((2, 7), "outflow"), ((7, 2), "slip"), ((3, 5), "slip"), ((2, 3), "noslip")]


@pytest.mark.parametrize("shape,bcname", _TINY)
def test_tiny_grids(shape, bcname):
    """Grids of one to a few cells: every stencil reaches into the ghost ring or wraps onto
    the cell itself (a 1 x 1 periodic grid is its own neighbour on all four sides; an axis one
    cell across must be periodic).  GPU and oracle agree over 5 Navier-Stokes steps."""
    nx, ny = shape
    p = _perturbed(nx, ny, seed=4, bc=BCSETS[bcname], mu=1e-3, Pr=0.72)
    g, o = _run_both(p, 5)
    for a, b in zip(g, o):
        assert _rel_linf(a, b) < 1e-10


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (3, 5)])
def test_tiny_periodic_grids_fp32_bulk_conserve(shape):
    """The FP32-bulk form on the same tiny periodic grids: finite states and totals kept to the
    double-float pair's roundoff."""
    nx, ny = shape
    p = _perturbed(nx, ny, seed=4, mu=1e-3, Pr=0.72)
    s = gks.Solver(p, gks.GKS_FP32_BULK)
    for _ in range(20):
        s.step(0.5)
    U = s.state()[0]
    s.close()
    assert np.all(np.isfinite(U))
    tot0, tot = p.U.sum(axis=(1, 2)), U.sum(axis=(1, 2))
    assert np.max(np.abs(tot - tot0) / np.abs(tot0).max()) < 1e-12


def test_riemann_ns_discontinuous():
    p = wl.riemann_2d(40, 36, seed=3, mu=1e-4, Pr=0.72)
    g, o = _run_both(p, 60)
    l1 = np.sum(np.abs(g[0][0] - o[0][0])) / np.sum(np.abs(o[0][0]))
    assert l1 < 1e-8


def test_riemann_euler_discontinuous():
    p = wl.riemann_2d(33, 41, seed=7, mu=0.0, Pr=1.0)
    g, o = _run_both(p, 60)
    l1 = np.sum(np.abs(g[0][0] - o[0][0])) / np.sum(np.abs(o[0][0]))
    assert l1 < 1e-8


def test_cavity():
    p = wl.cavity_2d(24)
    g, o = _run_both(p, 60)
    for a, b in zip(g, o):
        assert _rel_linf(a, b) < 1e-10


def test_density_wave_1d_to_t2():
    """Section 4.1 at 100 cells (nx by 1, periodic) to t = 2: GPU vs oracle, and vs the exact wave."""
    p = wl.density_wave_1d(100, seed=1)
    P = oracle.params(gamma=1.4, tau_eps=0.0)
    s = gks.Solver(p, gks.GKS_FP64, tau_eps=0.0)
    st = _state(p)
    n = 0
    while st.t < 2.0 * (1 - 1e-14):
        s.step(0.5, 2.0 - st.t)
        oracle.step2d(P, st, _oracle_bc(p), 0.5, 2.0 - st.t)
        st.t += 0  # time is kept by step2d
        n += 1
    U, Wx, Wy, t = s.state()
    s.close()
    assert t == pytest.approx(2.0, rel=1e-13)
    assert _rel_linf(U, st.U) < 1e-10
    exact = wl.density_wave_exact_avg(100, 2.0, p.meta["phi"])
    assert np.mean(np.abs(U[0, 0] - exact)) < 5e-5


def test_advance_matches_step():
    p = _perturbed(30, 22, seed=5, mu=1e-3, Pr=0.72)
    a = gks.Solver(p)
    b = gks.Solver(p)
    for _ in range(20):
        a.step(0.5)
    b.advance(20, 0.5)
    t, n = b.sync()
    assert n == 20
    Ua, Wxa, Wya, ta = a.state()
    Ub, Wxb, Wyb, tb = b.state()
    a.close()
    b.close()
    assert ta == tb
    assert np.array_equal(Ua, Ub) and np.array_equal(Wxa, Wxb) and np.array_equal(Wya, Wyb)


@pytest.mark.parametrize("prec", [gks.GKS_FP64, gks.GKS_FP32_BULK])
@pytest.mark.parametrize("nsteps", [6, 20])
def test_advance_matches_step_through_the_fallback(prec, nsteps):
    """On data where the positivity fallback fires (steps 3 and 5 in FP64) the replayed graphs
    (one-step graphs; a 16-step graph and four one-step ones) equal gks_step bit for bit."""
    quads = [(0.746, -0.312, 0.887, 0.312), (0.827, 0.438, -0.155, 0.861), (1.15, 0.953, 0.354, 0.494),
             (0.228, -0.698, -0.347, 1.304)]
    p = wl.riemann_2d(16, 80, quadrants=quads, mu=9.4e-4, Pr=0.72)
    p.bc = [(wl.BC_PERIODIC, 0.0, 0.0, 1.0)] * 4
    a = gks.Solver(p, prec)
    b = gks.Solver(p, prec)
    for _ in range(nsteps):
        a.step(0.5)
    b.advance(nsteps, 0.5)
    t, n = b.sync()
    assert n == nsteps
    Ua, Wxa, Wya, ta = a.state()
    Ub, Wxb, Wyb, tb = b.state()
    a.close()
    b.close()
    assert ta == tb
    assert np.array_equal(Ua, Ub) and np.array_equal(Wxa, Wxb) and np.array_equal(Wya, Wyb)


def test_advance_stops_at_t_end():
    p = wl.smooth_wave_2d(16, seed=2)
    s = gks.Solver(p, tau_eps=0.0)
    s.advance(500, 0.5, t_end=0.1)
    t, n = s.sync()
    s.close()
    assert t == pytest.approx(0.1, rel=1e-14) and 0 < n < 500


def test_device_state_round_trip():
    torch = pytest.importorskip("torch")
    p = _perturbed(21, 17, seed=9)
    s = gks.Solver(p)
    U = torch.zeros((4, p.ny, p.nx), dtype=torch.float64, device="cuda")
    Wx = torch.zeros((4, 2, p.ny, p.nx + 1), dtype=torch.float64, device="cuda")
    Wy = torch.zeros((4, 2, p.ny + 1, p.nx), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()  # the library works on its own stream
    gks.gks_get_state_device(s.h, U, Wx, Wy)
    assert np.array_equal(U.cpu().numpy(), p.U)
    assert np.array_equal(Wx.cpu().numpy(), p.Wx) and np.array_equal(Wy.cpu().numpy(), p.Wy)
    U2 = U * 1.0
    torch.cuda.synchronize()
    gks.gks_set_state_device(s.h, U2, Wx, Wy, 0.0)
    s.close()


def test_invalid_arguments():
    with pytest.raises(gks.GKSError) as e:
        gks.gks_create(0, 4, 1.0, 1.0, 1.4, 1.0, 0.0)
    assert e.value.status == gks.GKS_EINVAL
    with pytest.raises(gks.GKSError):
        gks.gks_create(4, 4, 1.0, 1.0, 0.9, 1.0, 0.0)
    with pytest.raises(gks.GKSError):
        gks.gks_create(4, 4, 1.0, 1.0, 1.4, 1.0, 0.0, bc=[wl.BC_PERIODIC, wl.BC_OUTFLOW, 0, 0])


def test_nonphysical_state_is_rejected_and_rolled_back():
    p = wl.smooth_wave_2d(12, seed=2)
    bad = p.U.copy()
    bad[0, 3, 4] = -1.0
    h = gks.gks_create(p.nx, p.ny, p.Lx, p.Ly, p.gamma, p.Pr, p.mu, p.bc)
    with pytest.raises(gks.GKSError) as e:
        gks.gks_set_state(h, bad, p.Wx, p.Wy)
    assert e.value.status == gks.GKS_ENONPHYSICAL
    gks.gks_destroy(h)
    # a strong rarefaction at an absurd CFL drives a cell non-physical; the step is not
    # taken and the state stays the one before it
    q = wl.riemann_2d(16, 16, quadrants=[(1.0, 5.0, 0.0, 1.0), (1.0, -5.0, 0.0, 1.0), (1.0, -5.0, 0.0, 1.0),
                                         (1.0, 5.0, 0.0, 1.0)], mu=0.0, Pr=1.0)
    s = gks.Solver(q)
    failed = False
    for _ in range(10):
        before = s.state()
        try:
            s.step(8.0)
        except gks.GKSError as err:
            assert err.status == gks.GKS_ENONPHYSICAL
            failed = True
            break
    assert failed
    U = np.zeros_like(q.U)
    st = gks.load().gks_get_state(s.h, gks._ptr(U), None, None, None)
    assert st == gks.GKS_ENONPHYSICAL
    assert np.array_equal(U, before[0])
    s.close()


def test_positivity_fallback_parity():
    """Seeded near-vacuum Riemann data on which the first-order fallback fires (steps 3 and 5):
    GPU and oracle take the same steps to roundoff."""
    quads = [(0.746, -0.312, 0.887, 0.312), (0.827, 0.438, -0.155, 0.861), (1.15, 0.953, 0.354, 0.494),
             (0.228, -0.698, -0.347, 1.304)]
    p = wl.riemann_2d(16, 80, quadrants=quads, mu=9.4e-4, Pr=0.72)
    p.bc = [(wl.BC_PERIODIC, 0.0, 0.0, 1.0)] * 4
    g, o = _run_both(p, 6)
    for a, b in zip(g, o):
        assert _rel_linf(a, b) < 1e-9


# ---- the characteristic-variable reconstruction (Section 4's choice for discontinuities) ----

@pytest.mark.parametrize("bcname", ["periodic", "noslip", "mixed"])
def test_characteristic_reconstruction_parity(bcname):
    p = _perturbed(37, 29, seed=1, bc=BCSETS[bcname])
    s = gks.Solver(p, characteristic=1)
    got = gks.gks_debug_recon(s.h, p.nx, p.ny)
    s.close()
    want = oracle.recon2d(_oracle_params(p, characteristic=1), _state(p), _oracle_bc(p))
    scale = np.abs(want).reshape(4, 6, -1).max(axis=2)[:, :, None, None] + 1e-300
    np.testing.assert_allclose(got / scale, want / scale, rtol=0, atol=1e-12)


@pytest.mark.parametrize("mu,Pr", [(0.0, 1.0), (1e-4, 0.72)])
def test_characteristic_riemann_parity(mu, Pr):
    p = wl.riemann_2d(40, 36, seed=3, mu=mu, Pr=Pr)
    g, o = _run_both(p, 60, P=oracle.params(gamma=p.gamma, mu=mu, Pr=Pr, characteristic=1), characteristic=1)
    l1 = np.sum(np.abs(g[0][0] - o[0][0])) / np.sum(np.abs(o[0][0]))
    assert l1 < 1e-8


def test_characteristic_smooth_wave_parity():
    p = wl.smooth_wave_2d(48, ny=40, seed=2)
    g, o = _run_both(p, 100, P=oracle.params(gamma=1.4, tau_eps=0.0, characteristic=1), tau_eps=0.0,
                     characteristic=1)
    for a, b in zip(g, o):
        assert _rel_linf(a, b) < 1e-10


def test_characteristic_fp32_bulk_within_budget():
    p = wl.riemann_2d(48, 40, seed=3, mu=1e-4, Pr=0.72)
    a = gks.Solver(p, gks.GKS_FP64, characteristic=1)
    b = gks.Solver(p, gks.GKS_FP32_BULK, characteristic=1)
    for s in (a, b):
        for _ in range(8):  # t ~ 0.03, within the workload's predictability horizon
            s.step(0.5)
    Ua, Ub = a.state()[0], b.state()[0]
    a.close()
    b.close()
    assert np.sum(np.abs(Ub[0] - Ua[0])) / np.sum(np.abs(Ua[0])) < 1e-5


@pytest.mark.parametrize("prec", [gks.GKS_FP64, gks.GKS_FP32_BULK])
def test_page_locked_host_arrays_round_trip_like_pageable_ones(prec):
    """gks_set_state / gks_get_state read and write page-locked host arrays in place (over the
    host link) and copy pageable ones through the staging buffer: the same state either way."""
    import torch
    p = wl.riemann_2d(70, 45, seed=3, mu=1e-4, Pr=0.72)

    def pinned_like(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t

    pins = [pinned_like(a) for a in (p.U, p.Wx, p.Wy)]
    out = []
    for host in ((p.U, p.Wx, p.Wy), tuple(t.numpy() for t in pins)):
        s = gks.Solver(p, prec)
        gks.gks_set_state(s.h, *host, 0.25)
        s.advance(3, 0.5)
        if host[0] is p.U:
            U, Wx, Wy, t = s.state()
        else:
            dst = [pinned_like(np.zeros_like(a)) for a in (p.U, p.Wx, p.Wy)]
            t = gks.gks_get_state(s.h, *(d.numpy() for d in dst))
            U, Wx, Wy = (d.numpy().copy() for d in dst)
        s.close()
        out.append((U, Wx, Wy, t))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
