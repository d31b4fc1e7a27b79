"""Domain decomposition of one grid into row slabs on the GPU (the partitioned step of gks.h,
Eq. finite over the whole grid): the slabs of one grid, advanced in one process with their
edge rows exchanged between the phases of each step, equal the single-grid run bit for bit
after 100 steps -- on a periodic axis (two and three slabs), between isothermal no-slip walls
and with outflow sides, in FP64 and in FP32-bulk.  The grids have power-of-two cell sizes, so
each slab's cell size equals the grid's exactly.  No kernel waits on another: the exchanges
are copies ordered by the host."""
import numpy as np
import pytest

from paper_1412_4489_gb300 import gks, parallel, workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 100


def _case(name):
    if name == "smooth_periodic":
        return wl.smooth_wave_2d(64, seed=2), {"tau_eps": 0.0}
    if name == "cavity_walls":
        p = wl.cavity_2d(32)
        p.bc[3] = (p.bc[3][0], 0.5, 0.0, p.bc[3][3])  # a faster lid: the flow moves within 100 steps
        return p, {}
    return wl.riemann_2d(64, seed=3, mu=1e-3, Pr=0.72), {}


@pytest.mark.parametrize("prec", [gks.GKS_FP64, gks.GKS_FP32_BULK])
@pytest.mark.parametrize("name,nslabs", [("smooth_periodic", 2), ("smooth_periodic", 3), ("cavity_walls", 2),
                                         ("riemann_outflow", 3)])
def test_slabs_equal_the_single_grid_bitwise(name, nslabs, prec):
    p, kw = _case(name)
    assert (p.Ly / p.ny) in (1 / 16, 1 / 32, 1 / 64) and (p.Lx / p.nx) in (1 / 16, 1 / 32, 1 / 64)
    single = gks.Solver(p, prec, **kw)
    dts = [single.step(0.5) for _ in range(STEPS)]
    U, Wx, Wy, t = single.state()
    single.close()
    run = parallel.LocalSlabs(p, nslabs, prec, **kw)
    dts_s = [run.step(0.5) for _ in range(STEPS)]
    Us, Wxs, Wys, ts = run.state()
    run.close()
    assert dts_s == dts and ts == t
    assert np.array_equal(Us, U), np.max(np.abs(Us - U))
    assert np.array_equal(Wxs, Wx) and np.array_equal(Wys, Wy)
    # and the state did move
    assert np.max(np.abs(U - p.U)) > 1e-4 * np.max(np.abs(p.U))


def test_exchange_sides_are_checked():
    p = wl.smooth_wave_2d(16, seed=2)
    bc = list(p.bc)
    bc[0] = (gks.GKS_BC_EXCHANGE, 0.0, 0.0, 1.0)
    bc[1] = (gks.GKS_BC_EXCHANGE, 0.0, 0.0, 1.0)
    with pytest.raises(gks.GKSError) as e:
        gks.gks_create(16, 16, 2.0, 2.0, 1.4, 1.0, 0.0, bc)
    assert e.value.status == gks.GKS_EINVAL
    s = gks.Solver(p, gks.GKS_FP64)
    buf = np.zeros(gks.gks_part_halo_bytes(s.h, gks.GKS_PART_STATE), dtype=np.uint8)
    with pytest.raises(gks.GKSError):  # a periodic side is not an exchange side
        gks.gks_part_get_edge(s.h, 2, gks.GKS_PART_STATE, buf)
    s.close()
