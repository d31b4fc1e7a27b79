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


@pytest.mark.parametrize("case", ["riemann_ns", "smooth_euler"])
def test_noalloc_matches_gks_step_on_two_calls(case):
    torch = pytest.importorskip("torch")
    if case == "riemann_ns":
        p = wl.riemann_2d(45, 38, seed=3, mu=1e-3, Pr=0.72)
        opts = gks.gks_default_options(gks.GKS_FP64)
    else:
        p = wl.smooth_wave_2d(40, ny=33, seed=2)
        opts = gks.gks_default_options(gks.GKS_FP64, tau_eps=0.0)
    # reference: a solver handle, two steps
    s = gks.Solver(p, gks.GKS_FP64, tau_eps=opts.tau_eps)
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
        dt = gks.gks_step_noalloc(p.nx, p.ny, p.Lx, p.Ly, p.gamma, p.Pr, p.mu, p.bc, opts, *cur, *out, 0.5)
        torch.cuda.synchronize()
        assert dt == pytest.approx(ref[k][0], rel=TOL)
        for got, want in zip(out, ref[k][1:]):
            _close(got.cpu().numpy(), want)
        cur = out


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
