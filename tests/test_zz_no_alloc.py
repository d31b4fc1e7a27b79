"""The allocation-free step (gks_step_noalloc) against the handle-based gks_step.

gks_step_noalloc serves callers that may not allocate device memory: it keeps the
scratch of a step in a static array of the library instead of calling cudaMalloc.  This
checks, through the C ABI, that two calls in a row -- each reusing the same static
scratch -- give the same states and time steps as gks_step on a solver handle, within
the FP64 tolerance of the other parity tests.  The file sorts last so that a failure here
stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

from paper_1412_4489_gb300 import gks, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _close(a, b):
    scale = np.max(np.abs(b))
    assert np.max(np.abs(a - b)) <= TOL * scale


def _case(case):
    """(problem, option overrides): periodic smooth wave, outflow Navier-Stokes Riemann data,
    the cavity's isothermal no-slip walls (whose images the update pass writes into the ghost
    ring), and the Riemann data with the characteristic reconstruction."""
    if case == "riemann_ns":
        return wl.riemann_2d(45, 38, seed=3, mu=1e-3, Pr=0.72), {}
    if case == "smooth_euler":
        return wl.smooth_wave_2d(40, ny=33, seed=2), {"tau_eps": 0.0}
    if case == "cavity_walls":
        p = wl.cavity_2d(36)
        # a lid faster than the workload's 0.15, so that two steps move the state visibly
        p.bc[3] = (p.bc[3][0], 0.5, 0.0, p.bc[3][3])
        return p, {}
    return wl.riemann_2d(37, 42, seed=3, mu=1e-3, Pr=0.72), {"characteristic": 1}


@pytest.mark.parametrize("case", ["riemann_ns", "smooth_euler", "cavity_walls", "riemann_characteristic"])
def test_noalloc_matches_gks_step_on_two_calls(case):
    torch = pytest.importorskip("torch")
    p, kw = _case(case)
    opts = gks.gks_default_options(gks.GKS_FP64, **kw)
    # reference: a solver handle, two steps
    s = gks.Solver(p, gks.GKS_FP64, **kw)
    ref = []
    for _ in range(2):
        dt = s.step(0.5)
        U, Wx, Wy, _ = s.state()
        ref.append((dt, U, Wx, Wy))
    s.close()
    # the same two steps through the allocation-free call, output of the first feeding the second
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    cur = [dev(p.U), dev(p.Wx), dev(p.Wy)]
    for k in range(2):
        out = [torch.full_like(x, float("nan")) for x in cur]
        before = [x.clone() for x in cur]
        dt = gks.gks_step_noalloc(p.nx, p.ny, p.Lx, p.Ly, p.gamma, p.Pr, p.mu, p.bc, opts, *cur, *out, 0.5)
        torch.cuda.synchronize()
        assert dt == pytest.approx(ref[k][0], rel=TOL)
        for got, want in zip(out, ref[k][1:]):
            _close(got.cpu().numpy(), want)
        # the inputs are read only
        for x, x0 in zip(cur, before):
            assert torch.equal(x, x0)
        cur = out
    # the state did move (a comparison of two unchanged states would prove nothing)
    assert np.max(np.abs(ref[1][1] - p.U)) > 1e-6 * np.max(np.abs(p.U))


def test_noalloc_fits_the_largest_padded_grid():
    """A single periodic column of 65,536 cells has the largest padded planes of any grid
    within the cell limit; it must fit the static scratch and match gks_step."""
    torch = pytest.importorskip("torch")
    p = wl.smooth_wave_2d(1, ny=65536, seed=2)
    opts = gks.gks_default_options(gks.GKS_FP64, tau_eps=0.0)
    s = gks.Solver(p, gks.GKS_FP64, tau_eps=0.0)
    dt_ref = s.step(0.5)
    U, Wx, Wy, _ = s.state()
    s.close()
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    cur = [dev(p.U), dev(p.Wx), dev(p.Wy)]
    out = [torch.full_like(x, float("nan")) for x in cur]
    dt = gks.gks_step_noalloc(p.nx, p.ny, p.Lx, p.Ly, p.gamma, p.Pr, p.mu, p.bc, opts, *cur, *out, 0.5)
    assert dt == pytest.approx(dt_ref, rel=TOL)
    for got, want in zip(out, (U, Wx, Wy)):
        _close(got.cpu().numpy(), want)


def test_noalloc_rejects_overlapping_outputs():
    torch = pytest.importorskip("torch")
    p = wl.smooth_wave_2d(16, seed=2)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    U, Wx, Wy = dev(p.U), dev(p.Wx), dev(p.Wy)
    outs = [U.clone(), Wx.clone(), Wy.clone()]
    for k, alias in ((0, U), (1, Wx), (2, Wy)):
        o = list(outs)
        o[k] = alias
        with pytest.raises(gks.GKSError) as e:
            gks.gks_step_noalloc(p.nx, p.ny, p.Lx, p.Ly, p.gamma, p.Pr, p.mu, p.bc, None, U, Wx, Wy, *o, 0.5)
        assert e.value.status == gks.GKS_EINVAL
        assert "overlap" in gks.gks_last_error(None)


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    p = wl.smooth_wave_2d(8, seed=2)
    U = torch.zeros((4, 300, 300), dtype=torch.float64, device="cuda")
    Wx = torch.zeros((4, 2, 300, 301), dtype=torch.float64, device="cuda")
    Wy = torch.zeros((4, 2, 301, 300), dtype=torch.float64, device="cuda")
    with pytest.raises(gks.GKSError) as e:
        gks.gks_step_noalloc(300, 300, 1.0, 1.0, 1.4, 1.0, 0.0, p.bc, None, U, Wx, Wy, U.clone(), Wx.clone(),
                             Wy.clone(), 0.5)
    assert e.value.status == gks.GKS_EINVAL
    assert "65,536 cells" in gks.gks_last_error(None)
