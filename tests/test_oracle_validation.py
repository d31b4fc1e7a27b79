"""Validation of the oracle on the paper's remaining analytic tests (Section 4.1, 4.2):

* the exact Riemann solver used as the Sod reference is pinned by the jump conditions
  (Rankine-Hugoniot across the shock, isentropic invariants across the rarefaction, continuous
  pressure and velocity across the contact);
* the oracle's Sod tube converges to that exact solution;
* the oracle's isotropic vortex errors after one period follow Table 2 (same order of
  magnitude, decreasing at better than second order between the first two meshes; the GPU
  tests take the finer meshes, where the order approaches the paper's 2.7-2.95).
"""
import math

import numpy as np
import pytest

import oracle
from exact_riemann import cell_average_density, sample, star_state
from paper_1412_4489_gb300 import workloads as wl

G = 1.4
SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def test_exact_riemann_jump_conditions():
    ps, us = star_state(SOD_L, SOD_R, G)
    # right shock: states either side and the shock speed satisfy Rankine-Hugoniot
    rr, ur, pr = SOD_R
    cr = math.sqrt(G * pr / rr)
    S = ur + cr * math.sqrt((G + 1) / (2 * G) * ps / pr + (G - 1) / (2 * G))
    rs, u2, p2 = sample(SOD_L, SOD_R, S - 1e-9, G)
    assert (u2, p2) == pytest.approx((us, ps), rel=1e-12)
    E = lambda r, u, p: p / (G - 1) + 0.5 * r * u * u
    for a, b in ((rr * (ur - S), rs * (us - S)),
                 (rr * ur * (ur - S) + pr, rs * us * (us - S) + ps),
                 ((E(rr, ur, pr) + pr) * ur - S * E(rr, ur, pr), (E(rs, us, ps) + ps) * us - S * E(rs, us, ps))):
        assert a == pytest.approx(b, rel=1e-10, abs=1e-12)
    # left rarefaction: entropy and the Riemann invariant u + 2c/(gamma-1) are constant through
    # the fan and into the star region
    rl, ul, pl = SOD_L
    inv = lambda r, u, p: (p / r ** G, u + 2 * math.sqrt(G * p / r) / (G - 1))
    ref = inv(rl, ul, pl)
    for s in np.linspace(-1.18, 0.5, 12):
        r, u, p = sample(SOD_L, SOD_R, s, G)
        if s < us:
            assert inv(r, u, p) == pytest.approx(ref, rel=1e-12)
    # contact: pressure and velocity continuous, density jumps
    a, b = sample(SOD_L, SOD_R, us - 1e-9, G), sample(SOD_L, SOD_R, us + 1e-9, G)
    assert a[1:] == pytest.approx(b[1:], rel=1e-12) and abs(a[0] - b[0]) > 0.1


def _sod_oracle(nx, tau_eps=0.05):
    p = wl.sod(nx)
    P = oracle.params(gamma=G, tau_eps=tau_eps)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
    bc = oracle.bcs([b[0] for b in p.bc])
    oracle.run2d(P, st, bc, 0.5, t_end=0.2)
    exact = cell_average_density(SOD_L, SOD_R, 0.5, 0.2, np.linspace(0, 1, nx + 1), G)
    return st, np.mean(np.abs(st.U[0, 0] - exact))


def test_oracle_sod_converges_to_the_exact_solution():
    """Section 4.2's Sod tube at t = 0.2: the L1 density error against the exact solution
    falls with the mesh (first order at the discontinuities) and stays small."""
    e = [_sod_oracle(n)[1] for n in (100, 200, 400)]
    assert e[0] < 1e-2 and e[1] < 0.7 * e[0] and e[2] < 0.7 * e[1], e


def test_oracle_isotropic_vortex_follows_table2():
    """Section 4.1 / Table 2 on the first two meshes (the oracle is slow beyond): errors after
    one period within [1/5, 2] of the paper's (the paper's weight constants and error definition
    are unstated), falling at better than second order."""
    table = np.loadtxt(__file__.replace("test_oracle_validation.py", "golden/table2_isotropic_vortex.txt"))
    P = oracle.params(gamma=G, tau_eps=0.0)
    e = []
    for n in (21, 41):
        p = wl.isotropic_vortex(n)
        st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
        oracle.run2d(P, st, oracle.bcs([oracle.BC_PERIODIC] * 4), 0.2, t_end=10.0)
        assert st.t == pytest.approx(10.0, rel=1e-14)
        d = st.U[0] - p.U[0]  # one period later the exact solution is the initial one
        e.append((np.mean(np.abs(d)), math.sqrt(np.mean(d * d))))
    e = np.array(e)
    assert np.all(e[:, 0] < 2 * table[:2, 1]) and np.all(e[:, 0] > table[:2, 1] / 5)
    assert np.all(e[:, 1] < 2 * table[:2, 3]) and np.all(e[:, 1] > table[:2, 3] / 5)
    order = math.log(e[0, 0] / e[1, 0]) / math.log(41 / 21)
    assert order > 2.0, order


def test_blast_wave_and_viscous_shock_tube_initial_data():
    """The Section 5 setups: exact totals of the piecewise-constant data, face point values
    on a break the mean of the two sides, reflecting / no-slip / symmetry boundaries."""
    g = 1.4
    b = wl.blast_wave(400)
    assert (b.nx, b.ny, b.Lx) == (400, 1, 100.0) and b.Ly == pytest.approx(0.25)
    # total energy p / (gamma - 1) over the three intervals, times the cell volume dx dy
    e = (1000.0 * 10 + 0.01 * 80 + 100.0 * 10) / (g - 1) / 100.0 * 400
    assert b.U[3].sum() == pytest.approx(e, rel=1e-13) and b.U[0].sum() == pytest.approx(400.0, rel=1e-14)
    assert np.all(b.U[1:3] == 0.0)
    assert b.Wx[3, :, 0, 40] == pytest.approx([(1000.0 + 0.01) / 2 / (g - 1)] * 2)  # the face at x = 10
    assert [k for k, *_ in b.bc] == [wl.BC_SLIPWALL, wl.BC_SLIPWALL, wl.BC_PERIODIC, wl.BC_PERIODIC]
    v = wl.viscous_shock_tube(300)
    assert (v.nx, v.ny, v.Lx, v.Ly) == (300, 150, 1.0, 0.5)
    assert v.mu == pytest.approx(1 / 200.0) and v.Pr == 0.73
    assert v.U[0, :, :150].min() == 120.0 and v.U[0, :, 150:].max() == pytest.approx(1.2)
    assert v.U[3, 0, 0] == pytest.approx(120.0 / g / (g - 1)) and v.Wx[0, :, 7, 150] == pytest.approx([60.6, 60.6])
    assert [k for k, *_ in v.bc] == [wl.BC_NOSLIP_ADIABATIC] * 3 + [wl.BC_SLIPWALL]
    assert all(w[1] == 0.0 and w[2] == 0.0 for w in v.bc)  # walls at rest
    # the oracle keeps both closed boxes' mass and energy to roundoff
    for p, n in ((b, 40), (wl.viscous_shock_tube(24), 20)):
        P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr, tau_eps=0.05)
        st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
        bc = oracle.bcs([k[0] for k in p.bc], [k[1:] for k in p.bc])
        for _ in range(n):
            rc, _ = oracle.step2d(P, st, bc, 0.5)
            assert rc == 0
        m0, m = p.U.reshape(4, -1).sum(axis=1), st.U.reshape(4, -1).sum(axis=1)
        assert abs(m[0] - m0[0]) <= 1e-13 * m0[0] and abs(m[3] - m0[3]) <= 1e-13 * m0[3]
