"""Grid-level pins of the oracle: what the paper and the mathematics fix for whole steps.

* free stream is preserved exactly (Eq. finite with identical face fluxes);
* mass, momentum and energy are conserved to roundoff on periodic grids and in a box of
  slip walls;
* the scheme commutes with the transposition x <-> y and the reflection x -> -x;
* data that do not depend on y reproduce the independent 1D scheme (one step, exactly);
* the density wave of Section 4.1 converges at third order (Table 1), in 1D and 2D.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1412_4489_gb300 import workloads as wl

G = math.sqrt(3.0) / 6.0
PER = [oracle.BC_PERIODIC] * 4


def _cons(rho, u, v, p, gamma):
    return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def _state(p):
    return oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)


def _perturbed(nx, ny, seed, gamma=1.4, amp=0.05):
    """A smooth periodic state with random small perturbations on cells and faces."""
    p = wl.smooth_wave_2d(nx, ny=ny, seed=seed, gamma=gamma)
    rng = np.random.default_rng(seed)
    st = _state(p)
    st.U *= 1 + amp * rng.uniform(-1, 1, size=st.U.shape) * np.array([1, 1, 1, 0.2])[:, None, None]
    st.Wx *= 1 + amp * rng.uniform(-1, 1, size=st.Wx.shape) * np.array([1, 1, 1, 0.2])[:, None, None, None]
    st.Wy *= 1 + amp * rng.uniform(-1, 1, size=st.Wy.shape) * np.array([1, 1, 1, 0.2])[:, None, None, None]
    # make periodic duplicate faces agree
    st.Wx[..., -1] = st.Wx[..., 0]
    st.Wy[:, :, -1, :] = st.Wy[:, :, 0, :]
    return st


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_free_stream(mu):
    gamma = 1.4
    w = _cons(0.8, 0.4, -0.7, 1.3, gamma)
    nx, ny = 7, 5
    U = np.broadcast_to(w[:, None, None], (4, ny, nx)).copy()
    Wx = np.broadcast_to(w[:, None, None, None], (4, 2, ny, nx + 1)).copy()
    Wy = np.broadcast_to(w[:, None, None, None], (4, 2, ny + 1, nx)).copy()
    st = oracle.State2D(nx, ny, 1.0, 0.8, U, Wx, Wy)
    P = oracle.params(gamma=gamma, mu=mu, Pr=0.72)
    oracle.step2d(P, st, oracle.bcs(PER), 0.5)
    assert np.array_equal(st.U, U)  # identical face fluxes cancel exactly
    for _ in range(20):
        oracle.step2d(P, st, oracle.bcs(PER), 0.5)
    np.testing.assert_allclose(st.U, U, rtol=1e-13)
    np.testing.assert_allclose(st.Wx, Wx, rtol=1e-13)
    np.testing.assert_allclose(st.Wy, Wy, rtol=1e-13)


@pytest.mark.parametrize("mu,Pr", [(0.0, 1.0), (2e-3, 0.72)])
def test_conservation_periodic(mu, Pr):
    st = _perturbed(12, 9, seed=4)
    P = oracle.params(gamma=1.4, mu=mu, Pr=Pr)
    tot0 = st.U.sum(axis=(1, 2))
    for _ in range(15):
        rc, _ = oracle.step2d(P, st, oracle.bcs(PER), 0.5)
        assert rc == 0
        np.testing.assert_allclose(st.U.sum(axis=(1, 2)), tot0, rtol=1e-13, atol=1e-13 * np.abs(tot0).max())


def test_conservation_riemann_periodic():
    p = wl.riemann_2d(16, 12, seed=3, mu=1e-3)
    st = _state(p)
    P = oracle.params(gamma=1.4, mu=1e-3, Pr=0.72)
    tot0 = st.U.sum(axis=(1, 2))
    for _ in range(10):
        rc, _ = oracle.step2d(P, st, oracle.bcs(PER), 0.5)
        assert rc == 0
    np.testing.assert_allclose(st.U.sum(axis=(1, 2)), tot0, rtol=1e-13, atol=1e-13 * np.abs(tot0).max())


def test_slip_wall_box_conserves_mass_and_energy():
    p = wl.riemann_2d(10, 8, seed=9, mu=0.0)
    st = _state(p)
    P = oracle.params(gamma=1.4)
    bc = oracle.bcs([oracle.BC_SLIPWALL] * 4)
    tot0 = st.U.sum(axis=(1, 2))
    for _ in range(10):
        assert oracle.step2d(P, st, bc, 0.4)[0] == 0
    tot = st.U.sum(axis=(1, 2))
    assert tot[0] == pytest.approx(tot0[0], rel=1e-13)
    assert tot[3] == pytest.approx(tot0[3], rel=1e-13)


def test_cavity_at_rest_stays_at_rest():
    p = wl.cavity_2d(8, lid=0.0)
    st = _state(p)
    P = oracle.params(gamma=p.gamma, mu=p.mu, Pr=p.Pr)
    bc = oracle.bcs([b[0] for b in p.bc], [b[1:] for b in p.bc])
    for _ in range(5):
        assert oracle.step2d(P, st, bc, 0.5)[0] == 0
    np.testing.assert_allclose(st.U, p.U, rtol=1e-13, atol=1e-14)


def _transpose(st):
    U = st.U.transpose(0, 2, 1)[[0, 2, 1, 3]]
    Wx = st.Wy.transpose(0, 1, 3, 2)[[0, 2, 1, 3]]
    Wy = st.Wx.transpose(0, 1, 3, 2)[[0, 2, 1, 3]]
    return oracle.State2D(st.ny, st.nx, st.Ly, st.Lx, U, Wx, Wy)


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_transpose_symmetry(mu):
    st = _perturbed(10, 7, seed=6)
    st.Ly = 1.5
    tr = _transpose(st)
    P = oracle.params(gamma=1.4, mu=mu, Pr=0.72)
    for _ in range(4):
        oracle.step2d(P, st, oracle.bcs(PER), 0.5)
        oracle.step2d(P, tr, oracle.bcs(PER), 0.5)
    back = _transpose(tr)
    np.testing.assert_allclose(back.U, st.U, rtol=1e-12)
    np.testing.assert_allclose(back.Wx, st.Wx, rtol=1e-12)
    np.testing.assert_allclose(back.Wy, st.Wy, rtol=1e-12)


def _reflect_x(st):
    sgn = np.array([1, -1, 1, 1])[:, None, None]
    U = st.U[:, :, ::-1] * sgn
    Wx = st.Wx[:, :, :, ::-1] * sgn[:, None]
    Wy = st.Wy[:, ::-1, :, ::-1] * sgn[:, None]  # x-Gauss points swap under x -> -x
    return oracle.State2D(st.nx, st.ny, st.Lx, st.Ly, U.copy(), Wx.copy(), Wy.copy())


@pytest.mark.parametrize("kinds", [PER, [oracle.BC_OUTFLOW] * 4])
def test_reflection_symmetry(kinds):
    st = _perturbed(9, 8, seed=2)
    rf = _reflect_x(st)
    P = oracle.params(gamma=1.4, mu=1e-3, Pr=0.72)
    for _ in range(4):
        oracle.step2d(P, st, oracle.bcs(kinds), 0.5)
        oracle.step2d(P, rf, oracle.bcs(kinds), 0.5)
    back = _reflect_x(rf)
    np.testing.assert_allclose(back.U, st.U, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(back.Wx, st.Wx, rtol=1e-12, atol=1e-13)


def _minmod(a, b):
    return np.where(a * b > 0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_y_uniform_data_reproduce_the_1d_scheme(mu):
    """One step of the 2D oracle on an nx-by-1 periodic grid with V = 0 equals one step of the
    independent 1D oracle (K1 = K + 1 absorbs v into the internal degrees of freedom).

    The y-face point values are set to those of the cell's limited one-sided polynomial
    U_1 (x) at x = -/+ sqrt(3)/6 dx, so that the 2D reconstruction has a3 = a5 = a6 = 0."""
    nx, gamma = 24, 1.4
    p = wl.density_wave_1d(nx, phi=0.37)
    U1, W1 = wl.density_wave_1d_layout(p)
    dx = p.Lx / nx
    Um, Up = np.roll(U1, 1, axis=1), np.roll(U1, -1, axis=1)
    Wm, Wp = W1[:, :-1], W1[:, 1:]
    a3 = _minmod(3 * (U1 + Um - 2 * Wm) / dx ** 2, 3 * (U1 + Up - 2 * Wp) / dx ** 2)
    a2 = _minmod(-2 * (Wm - U1) / dx + a3 * dx / 6, 2 * (Wp - U1) / dx - a3 * dx / 6)
    st = _state(p)
    for g, s in ((0, -1), (1, 1)):
        for j in range(2):
            st.Wy[[0, 1, 3], g, j, :] = U1 + s * G * dx * a2
            st.Wy[2, g, j, :] = 0.0
    P = oracle.params(gamma=gamma, mu=mu, Pr=0.72 if mu else 1.0)
    rc2, dt2 = oracle.step2d(P, st, oracle.bcs(PER), 0.5)
    rc1, dt1 = oracle.step1d(P, nx, p.Lx, U1, W1, 0.5)
    assert rc1 == rc2 == 0
    assert dt2 == pytest.approx(dt1, rel=1e-15)
    np.testing.assert_allclose(st.U[[0, 1, 3], 0], U1, rtol=1e-13)
    np.testing.assert_allclose(st.U[2], 0.0, atol=1e-15)
    for g in range(2):
        np.testing.assert_allclose(st.Wx[[0, 1, 3], g, 0], W1, rtol=1e-13)


def _wave_errors_1d(P, cells, cfl=0.2):
    out = []
    for nx in cells:
        p = wl.density_wave_1d(nx, phi=0.0)
        U1, W1 = wl.density_wave_1d_layout(p)
        oracle.run1d(P, nx, 2.0, U1, W1, cfl, 2.0)
        ex = wl.density_wave_exact_avg(nx, 2.0, 0.0)
        out.append((np.mean(np.abs(U1[0] - ex)), math.sqrt(np.mean((U1[0] - ex) ** 2))))
    return np.array(out)


def test_density_wave_third_order_1d():
    """Section 4.1 / Table 1 in the Euler limit of the collision time (epsilon = 0)."""
    e = _wave_errors_1d(oracle.params(tau_eps=0.0), [25, 50, 100, 200])
    orders = np.log2(e[:-1, 0] / e[1:, 0])
    assert np.all(orders > 2.9), orders
    table = np.loadtxt(__file__.replace("test_oracle_solver.py", "golden/table1_density_wave.txt"))
    paper_orders = table[1:, 2]
    assert np.all(paper_orders > 2.8)  # the order the paper reports, which ours matches
    # our error constant: within 20x of Table 1 at 50..200 cells (the paper's weights are unstated)
    assert np.all(e[1:, 0] < 20 * table[:3, 1])


def test_paper_inviscid_tau_limits_smooth_order():
    """With the inviscid tau = 0.05 dt of Section 4 the epsilon dt collision time adds an O(dt)
    heat conduction: the smooth wave converges at first order only.  This is why the accuracy
    workloads use epsilon = 0 (a reading recorded with the design)."""
    e = _wave_errors_1d(oracle.params(tau_eps=0.05), [50, 100, 200])
    orders = np.log2(e[:-1, 0] / e[1:, 0])
    assert np.all(orders < 1.8), orders


def test_smooth_wave_2d_converges():
    P = oracle.params(gamma=1.4, tau_eps=0.0)
    errs = []
    for n in (16, 32, 64):
        p = wl.smooth_wave_2d(n, seed=2)
        st = _state(p)
        oracle.run2d(P, st, oracle.bcs(PER), 0.5, t_end=1.0)  # one period along x + y
        errs.append(np.mean(np.abs(st.U[0] - p.U[0])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # third order, approached from above on these meshes (3.6, 3.4 with C = 10)
    assert np.all(orders > 2.7) and abs(orders[1] - 3.0) < abs(orders[0] - 3.0) + 0.2, orders


def test_positivity_fallback_rescues_a_near_vacuum_riemann_problem():
    """Seeded four-quadrant data whose high-order update drives a cell to p < 0 in the second
    step (a near-vacuum forms at a quadrant interface).  With the first-order fallback at the
    faces of such cells the run continues, stays physical and conserves mass on a periodic grid."""
    quads = [(0.746, -0.312, 0.887, 0.312), (0.827, 0.438, -0.155, 0.861), (1.15, 0.953, 0.354, 0.494),
             (0.228, -0.698, -0.347, 1.304)]
    p = wl.riemann_2d(16, 80, quadrants=quads, mu=9.4e-4, Pr=0.72)
    st = _state(p)
    P = oracle.params(gamma=1.4, mu=9.4e-4, Pr=0.72)
    tot0 = st.U[0].sum()
    for _ in range(6):
        rc, _ = oracle.step2d(P, st, oracle.bcs(PER), 0.5)
        assert rc == 0
        pr = 0.4 * (st.U[3] - 0.5 * (st.U[1] ** 2 + st.U[2] ** 2) / st.U[0])
        assert st.U[0].min() > 0 and pr.min() > 0
    assert st.U[0].sum() == pytest.approx(tot0, rel=1e-13)


@pytest.mark.parametrize("kind", [oracle.BC_SLIPWALL, oracle.BC_NOSLIP_ISOTHERMAL, oracle.BC_NOSLIP_ADIABATIC])
def test_closed_box_conserves_mass_and_the_adiabatic_energy(kind):
    """A box closed by four resting walls: no mass crosses a wall face, so the total mass is
    conserved to roundoff for every wall kind; slip and adiabatic walls also let no energy
    through (an isothermal wall exchanges heat).  The initial flow runs into the walls."""
    p = wl.smooth_wave_2d(18, ny=14, seed=4)
    P = oracle.params(gamma=1.4, mu=2e-3, Pr=0.72, tau_eps=0.05)
    st = _state(p)
    bc = oracle.bcs([kind] * 4, [(0.0, 0.0, 0.9)] * 4)
    tot0 = st.U.sum(axis=(1, 2))
    for _ in range(25):
        assert oracle.step2d(P, st, bc, 0.5)[0] == 0
    tot = st.U.sum(axis=(1, 2))
    assert abs(tot[0] - tot0[0]) < 1e-13 * tot0[0]
    if kind != oracle.BC_NOSLIP_ISOTHERMAL:
        assert abs(tot[3] - tot0[3]) < 1e-13 * tot0[3]
    else:
        assert abs(tot[3] - tot0[3]) > 1e-6 * tot0[3]  # heat drawn by the walls at T_w = 0.9 < T
    # the walls stop the flow that runs into them: momentum is not conserved
    assert np.all(np.abs(tot[1:3] - tot0[1:3]) > 1e-3 * np.abs(tot0[1:3]))


def test_adiabatic_moving_wall_does_work():
    """A moving adiabatic lid: the energy entering through it equals the work of the shear on
    the lid, u_w times the tangential momentum entering (no heat through the wall)."""
    p = wl.cavity_2d(16)
    P = oracle.params(gamma=1.4, mu=0.01, Pr=0.72)
    st = _state(p)
    wall = (0.0, 0.0, 1.0)
    bc = oracle.bcs([oracle.BC_NOSLIP_ADIABATIC] * 4, [wall, wall, wall, (0.3, 0.0, 1.0)])
    tot0 = st.U.sum(axis=(1, 2))
    for _ in range(20):
        assert oracle.step2d(P, st, bc, 0.5)[0] == 0
    d = st.U.sum(axis=(1, 2)) - tot0
    assert abs(d[0]) < 1e-13 * tot0[0]
    # x-momentum enters through the lid (the only moving wall) and friction on the other walls
    # removes some; the energy gained is the lid's work, which is positive
    assert d[3] > 0 and d[1] > 0


def _isobaric_mode_decay_rate(Pr, mu=0.01, nx=32, eps=1e-3, t_end=2.0, gamma=1.4):
    """Decay rate of an isobaric temperature mode T = 1 + eps sin(2 pi x) (p = 1, at rest) on a
    periodic nx-by-1 grid (exact cell averages and point values)."""
    dx, k = 1.0 / nx, 2.0 * np.pi
    rho = lambda x: 1.0 / (1.0 + eps * np.sin(k * x))
    xg, wg = np.polynomial.legendre.leggauss(6)
    xc = (np.arange(nx) + 0.5) * dx
    U = np.zeros((4, 1, nx))
    U[0, 0] = (rho(xc[:, None] + 0.5 * dx * xg[None, :]) * wg).sum(axis=1) / 2
    U[3] = 1.0 / (gamma - 1)
    Wx = np.zeros((4, 2, 1, nx + 1))
    Wx[0] = rho(np.arange(nx + 1) * dx)[None, None, :]
    Wx[3] = 1.0 / (gamma - 1)
    Wy = np.zeros((4, 2, 2, nx))
    Wy[0] = rho(xc[None, :] + np.array([-1.0, 1.0])[:, None] * dx * math.sqrt(3) / 6)[:, None, :]
    Wy[3] = 1.0 / (gamma - 1)
    P = oracle.params(gamma=gamma, mu=mu, Pr=Pr)
    st = oracle.State2D(nx, 1, 1.0, dx, U, Wx, Wy)
    bc = oracle.bcs([0, 0, 0, 0])

    def amplitude():
        T = (gamma - 1) * (st.U[3, 0] - 0.5 * st.U[1, 0] ** 2 / st.U[0, 0]) / st.U[0, 0]
        return 2 * abs(np.fft.rfft(T - T.mean())[1]) / nx

    a0 = amplitude()
    while st.t < t_end:
        rc, _ = oracle.step2d(P, st, bc, 0.5, dt_max=t_end - st.t, viscous_dt=1)
        assert rc == 0
    return math.log(a0 / amplitude()) / st.t


def test_prandtl_fix_gives_fouriers_law():
    """The Prandtl-number correction (energy flux += (1/Pr - 1) q) pinned by physics instead of
    the paper: an isobaric temperature mode decays at chi k^2 with chi = kappa / (rho c_p) =
    mu / (Pr rho) (Fourier's law with kappa = mu c_p / Pr), so the rate must scale as 1/Pr.
    Measured: 1.02 chi k^2 at both Pr = 1 (the plain BGK conductivity) and Pr = 0.72, at 16, 32
    and 64 cells alike; their ratio 1.3868 against 1/0.72 = 1.3889."""
    k2 = (2 * math.pi) ** 2
    r1, r72 = _isobaric_mode_decay_rate(1.0), _isobaric_mode_decay_rate(0.72)
    assert r1 == pytest.approx(0.01 * k2, rel=0.05)
    assert r72 == pytest.approx(0.01 / 0.72 * k2, rel=0.05)
    assert r72 / r1 == pytest.approx(1 / 0.72, rel=0.01)


def _shear_mode_decay_rate(Pr, mu=0.01, nx=32, eps=1e-3, t_end=2.0, gamma=1.4):
    """Decay rate of a transverse shear mode V = eps sin(2 pi x) (rho = 1, p = 1) on a periodic
    nx-by-1 grid (exact cell averages and point values)."""
    dx, k = 1.0 / nx, 2.0 * np.pi
    v = lambda x: eps * np.sin(k * x)
    xg, wg = np.polynomial.legendre.leggauss(6)
    xc = (np.arange(nx) + 0.5) * dx
    pts = xc[:, None] + 0.5 * dx * xg[None, :]
    U = np.zeros((4, 1, nx))
    U[0] = 1.0
    U[2, 0] = (v(pts) * wg).sum(axis=1) / 2
    U[3, 0] = 1.0 / (gamma - 1) + 0.5 * (v(pts) ** 2 * wg).sum(axis=1) / 2
    state = lambda vv: np.stack([np.ones_like(vv), np.zeros_like(vv), vv, 1.0 / (gamma - 1) + 0.5 * vv * vv])
    Wx = state(v(np.arange(nx + 1) * dx))[:, None, None, :].repeat(2, axis=1)
    Wy = state(v(xc[None, :] + np.array([-1.0, 1.0])[:, None] * dx * math.sqrt(3) / 6))[:, :, None, :].repeat(2, axis=2)
    P = oracle.params(gamma=gamma, mu=mu, Pr=Pr)
    st = oracle.State2D(nx, 1, 1.0, dx, U, np.ascontiguousarray(Wx), np.ascontiguousarray(Wy))
    bc = oracle.bcs([0, 0, 0, 0])
    amplitude = lambda: 2 * abs(np.fft.rfft(st.U[2, 0] / st.U[0, 0])[1]) / nx
    a0 = amplitude()
    while st.t < t_end:
        rc, _ = oracle.step2d(P, st, bc, 0.5, dt_max=t_end - st.t, viscous_dt=1)
        assert rc == 0
    return math.log(a0 / amplitude()) / st.t


def test_viscous_collision_time_gives_the_shear_viscosity():
    """tau = mu / p (Section 4) pinned by physics: a transverse shear mode decays at nu k^2 =
    mu k^2 / rho (measured within 1e-4 at 32 and 64 cells), and the Prandtl correction, which
    touches only the energy flux, leaves it unchanged."""
    k2 = (2 * math.pi) ** 2
    r1, r72 = _shear_mode_decay_rate(1.0), _shear_mode_decay_rate(0.72)
    assert r1 == pytest.approx(0.01 * k2, rel=1e-3)
    assert r72 == pytest.approx(r1, rel=1e-3)


def test_isothermal_walls_conduct_fouriers_heat_flux():
    """The isothermal no-slip wall image pinned by physics: gas at rest between walls at
    T = 1.2 and 0.8 (mu = 0.05, Pr = 1, 16 cells) relaxes to steady conduction in which every
    face, the two wall faces included, carries the same energy flux, the bulk conductivity is
    mu c_p (Fourier's law for the BGK gas), and the linear bulk profile meets the walls at their
    temperatures (measured: conductivity within 1.3e-4, wall values within 1.5e-3)."""
    g, nx, mu, T1, T2 = 1.4, 16, 0.05, 1.2, 0.8
    dx = 1.0 / nx
    U = np.zeros((4, 1, nx))
    U[0] = 1.0
    U[3] = 1.0 / (g - 1)
    Wx = np.ascontiguousarray(np.broadcast_to(U[:, None, :, :1], (4, 2, 1, nx + 1)))
    Wy = np.ascontiguousarray(np.broadcast_to(U[:, None, :1, :], (4, 2, 2, nx)))
    P = oracle.params(gamma=g, mu=mu, Pr=1.0)
    st = oracle.State2D(nx, 1, 1.0, dx, U, Wx, Wy)
    bc = oracle.bcs([3, 3, 0, 0], [(0.0, 0.0, T1), (0.0, 0.0, T2), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0)])
    while st.t < 60.0:  # four conduction times L^2 rho c_v / kappa
        rc, _ = oracle.step2d(P, st, bc, 0.5, viscous_dt=1)
        assert rc == 0
    dt = oracle.dt2d(P, st, 0.5, viscous_dt=1)
    Fx, _, _, _ = oracle.flux2d(P, st, bc, dt)
    q = Fx[3, 0] / dt
    assert np.ptp(q) <= 1e-3 * abs(q.mean()), q
    assert np.all(Fx[0, 0, [0, -1]] == 0.0)  # impermeable walls
    T = (g - 1) * (st.U[3, 0] - 0.5 * st.U[1, 0] ** 2 / st.U[0, 0]) / st.U[0, 0]
    x = (np.arange(nx) + 0.5) * dx
    slope, icpt = np.polyfit(x[nx // 4:3 * nx // 4], T[nx // 4:3 * nx // 4], 1)
    assert -q.mean() / slope == pytest.approx(mu * g / (g - 1), rel=1e-2)
    assert icpt == pytest.approx(T1, abs=1e-2) and icpt + slope == pytest.approx(T2, abs=1e-2)
    assert np.abs(st.U[1, 0] / st.U[0, 0]).max() < 1e-2


def test_moving_isothermal_wall_gives_couette_flow():
    """The moving no-slip (isothermal) wall pinned by plane Couette flow: walls at T = 1, the
    one at x = 1 sliding at V_w = 0.1 (mu = 0.05, Pr = 1, 16 cells).  Steady state: the shear
    stress is the same through every face, walls included, and equals mu dV/dx of a linear
    profile that meets both wall velocities; the wall's work mu V_w^2 / L leaves as heat, half
    through each wall, so the total energy flux is -mu V_w^2 / (2 L) through every face
    (measured: stress uniform to 1e-14, mu dV/dx and the wall velocities to 1e-5)."""
    g, nx, mu, Vw = 1.4, 16, 0.05, 0.1
    dx = 1.0 / nx
    U = np.zeros((4, 1, nx))
    U[0] = 1.0
    U[3] = 1.0 / (g - 1)
    Wx = np.ascontiguousarray(np.broadcast_to(U[:, None, :, :1], (4, 2, 1, nx + 1)))
    Wy = np.ascontiguousarray(np.broadcast_to(U[:, None, :1, :], (4, 2, 2, nx)))
    P = oracle.params(gamma=g, mu=mu, Pr=1.0)
    st = oracle.State2D(nx, 1, 1.0, dx, U, Wx, Wy)
    bc = oracle.bcs([3, 3, 0, 0], [(0.0, 0.0, 1.0), (0.0, Vw, 1.0), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0)])
    while st.t < 80.0:  # four viscous times L^2 / nu
        rc, _ = oracle.step2d(P, st, bc, 0.5, viscous_dt=1)
        assert rc == 0
    dt = oracle.dt2d(P, st, 0.5, viscous_dt=1)
    Fx, _, _, _ = oracle.flux2d(P, st, bc, dt)
    stress, energy = Fx[2, 0] / dt, Fx[3, 0] / dt
    V = st.U[2, 0] / st.U[0, 0]
    x = (np.arange(nx) + 0.5) * dx
    slope, icpt = np.polyfit(x[nx // 4:3 * nx // 4], V[nx // 4:3 * nx // 4], 1)
    assert np.ptp(stress) <= 1e-8 * abs(stress.mean())
    assert -stress.mean() == pytest.approx(mu * slope, rel=1e-3)
    assert icpt == pytest.approx(0.0, abs=1e-3 * Vw) and icpt + slope == pytest.approx(Vw, rel=1e-3)
    assert np.all(Fx[0, 0, [0, -1]] == 0.0)
    assert energy == pytest.approx(np.full(nx + 1, -mu * Vw * Vw / 2), rel=1e-2)


def test_moving_adiabatic_wall_sends_its_work_to_the_isothermal_wall():
    """The adiabatic no-slip wall pinned by Couette flow: the sliding wall at x = 1 adiabatic
    (V_w = 0.1), the fixed one at x = 0 isothermal (T = 1).  No heat crosses the adiabatic wall,
    so the whole work mu V_w^2 / L leaves through the isothermal one: the total energy flux is
    -mu V_w^2 / L through every face, the stress mu dV/dx, and the temperature peaks at the
    adiabatic wall with zero slope (measured: flux and stress to 1e-5)."""
    g, nx, mu, Vw = 1.4, 16, 0.05, 0.1
    dx = 1.0 / nx
    U = np.zeros((4, 1, nx))
    U[0] = 1.0
    U[3] = 1.0 / (g - 1)
    Wx = np.ascontiguousarray(np.broadcast_to(U[:, None, :, :1], (4, 2, 1, nx + 1)))
    Wy = np.ascontiguousarray(np.broadcast_to(U[:, None, :1, :], (4, 2, 2, nx)))
    P = oracle.params(gamma=g, mu=mu, Pr=1.0)
    st = oracle.State2D(nx, 1, 1.0, dx, U, Wx, Wy)
    bc = oracle.bcs([3, 4, 0, 0], [(0.0, 0.0, 1.0), (0.0, Vw, 1.0), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0)])
    while st.t < 120.0:  # the temperature relaxes over rho c_v L^2 / kappa, longer than L^2 / nu
        rc, _ = oracle.step2d(P, st, bc, 0.5, viscous_dt=1)
        assert rc == 0
    dt = oracle.dt2d(P, st, 0.5, viscous_dt=1)
    Fx, _, _, _ = oracle.flux2d(P, st, bc, dt)
    stress, energy = Fx[2, 0] / dt, Fx[3, 0] / dt
    V = st.U[2, 0] / st.U[0, 0]
    T = (g - 1) * (st.U[3, 0] - 0.5 * (st.U[1, 0] ** 2 + st.U[2, 0] ** 2) / st.U[0, 0]) / st.U[0, 0]
    x = (np.arange(nx) + 0.5) * dx
    slope = np.polyfit(x[nx // 4:3 * nx // 4], V[nx // 4:3 * nx // 4], 1)[0]
    assert -stress.mean() == pytest.approx(mu * slope, rel=1e-3) and np.ptp(stress) <= 1e-8 * abs(stress.mean())
    assert energy == pytest.approx(np.full(nx + 1, -mu * Vw * Vw), rel=1e-2)
    assert np.all(np.diff(T) > 0) and (T[-1] - T[-2]) < 0.1 * (T[1] - T[0])


def _mirror_symmetric_wave(nx, L, gamma=1.4):
    """rho = 1 + 0.2 cos(2 pi x), u = 0.3 sin(2 pi x), p = 1 + 0.1 cos(2 pi x), v = 0 on [0, L]
    (nx-by-1, exact cell averages and point values): mirror symmetric about x = 0 and 0.5."""
    dx = L / nx
    cons = lambda x: np.stack([1.0 + 0.2 * np.cos(2 * np.pi * x), (1.0 + 0.2 * np.cos(2 * np.pi * x)) * 0.3 * np.sin(2 * np.pi * x),
                               0.0 * x, (1.0 + 0.1 * np.cos(2 * np.pi * x)) / (gamma - 1)
                               + 0.5 * (1.0 + 0.2 * np.cos(2 * np.pi * x)) * (0.3 * np.sin(2 * np.pi * x)) ** 2])
    xg, wg = np.polynomial.legendre.leggauss(6)
    xc = (np.arange(nx) + 0.5) * dx
    U = (cons(xc[:, None] + 0.5 * dx * xg[None, :]) * wg).sum(axis=-1)[:, None, :] / 2
    Wx = np.repeat(cons(np.arange(nx + 1) * dx)[:, None, None, :], 2, axis=1)
    Wy = np.repeat(cons(xc[None, :] + np.array([-1.0, 1.0])[:, None] * dx * math.sqrt(3) / 6)[:, :, None, :], 2, axis=2)
    return oracle.State2D(nx, 1, L, dx, np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy))


@pytest.mark.parametrize("mu", [0.0, 1e-3])
def test_slip_walls_are_symmetry_planes(mu):
    """The slip-wall image pinned by symmetry: data mirror symmetric about x = 0 and x = 0.5 on
    the periodic [0, 1] evolve exactly like the half domain [0, 0.5] closed by slip walls (60
    steps, Euler and Navier-Stokes; measured equal to 1e-15)."""
    P = oracle.params(gamma=1.4, mu=mu, Pr=0.72 if mu else 1.0, tau_eps=0.05 if mu else 0.0)
    full, half = _mirror_symmetric_wave(64, 1.0), _mirror_symmetric_wave(32, 0.5)
    for _ in range(60):
        assert oracle.step2d(P, full, oracle.bcs([0, 0, 0, 0]), 0.5)[0] == 0
        assert oracle.step2d(P, half, oracle.bcs([2, 2, 0, 0]), 0.5)[0] == 0
    assert half.t == pytest.approx(full.t, rel=1e-14)
    # one scale for all variables: rho V stays at roundoff level (v = 0 by symmetry)
    assert np.max(np.abs(full.U[:, :, :32] - half.U)) < 1e-13 * np.abs(full.U).max()


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_acoustic_wave_travels_at_the_speed_of_sound(gamma):
    """The Euler limit pinned by the sound speed: a right-going acoustic wave (rho' = 1e-4 sin 2 pi x
    about rho = p = 1, u' = c rho', p' = c^2 rho') on a periodic 32-by-1 grid moves at
    sqrt(gamma p / rho); that needs the internal degrees of freedom K = (4 - 2 gamma)/(gamma - 1)
    of the 2D Maxwellian (measured within 1e-5 at 32 cells, 6e-7 at 64)."""
    nx, eps, k, t_end = 32, 1e-4, 2 * math.pi, 0.5
    dx, c = 1.0 / nx, math.sqrt(gamma)

    def cons(x):
        r = 1.0 + eps * np.sin(k * x)
        u = c * eps * np.sin(k * x)
        p = 1.0 + c * c * eps * np.sin(k * x)
        return np.stack([r, r * u, 0.0 * x, p / (gamma - 1) + 0.5 * r * u * u])

    xg, wg = np.polynomial.legendre.leggauss(6)
    xc = (np.arange(nx) + 0.5) * dx
    U = (cons(xc[:, None] + 0.5 * dx * xg[None, :]) * wg).sum(axis=-1)[:, None, :] / 2
    Wx = np.repeat(cons(np.arange(nx + 1) * dx)[:, None, None, :], 2, axis=1)
    Wy = np.repeat(cons(xc[None, :] + np.array([-1.0, 1.0])[:, None] * dx * math.sqrt(3) / 6)[:, :, None, :], 2, axis=2)
    st = oracle.State2D(nx, 1, 1.0, dx, np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy))
    P = oracle.params(gamma=gamma, tau_eps=0.0)
    phase0 = np.angle(np.fft.rfft(st.U[0, 0])[1])
    while st.t < t_end:
        assert oracle.step2d(P, st, oracle.bcs([0, 0, 0, 0]), 0.5, dt_max=t_end - st.t)[0] == 0
    moved = (phase0 - np.angle(np.fft.rfft(st.U[0, 0])[1])) % (2 * math.pi)
    assert moved / (k * st.t) == pytest.approx(c, rel=1e-4)


def _acoustic_damping(nx, gamma, Pr, mu=0.01, eps=1e-4, t_end=2.0):
    """(measured, Navier-Stokes) temporal damping rate of a right-going acoustic wave on a
    periodic nx-by-1 grid.  The BGK gas with N = 2/(gamma - 1) degrees of freedom has the
    longitudinal viscosity 2 mu (N - 1)/N, so the rate is k^2/(2 rho) (2 mu (N - 1)/N +
    (gamma - 1) mu / Pr)."""
    dx, k, c = 1.0 / nx, 2 * math.pi, math.sqrt(gamma)

    def cons(x):
        r = 1.0 + eps * np.sin(k * x)
        u = c * eps * np.sin(k * x)
        p = 1.0 + c * c * eps * np.sin(k * x)
        return np.stack([r, r * u, 0.0 * x, p / (gamma - 1) + 0.5 * r * u * u])

    xg, wg = np.polynomial.legendre.leggauss(6)
    xc = (np.arange(nx) + 0.5) * dx
    U = (cons(xc[:, None] + 0.5 * dx * xg[None, :]) * wg).sum(axis=-1)[:, None, :] / 2
    Wx = np.repeat(cons(np.arange(nx + 1) * dx)[:, None, None, :], 2, axis=1)
    Wy = np.repeat(cons(xc[None, :] + np.array([-1.0, 1.0])[:, None] * dx * math.sqrt(3) / 6)[:, :, None, :], 2, axis=2)
    st = oracle.State2D(nx, 1, 1.0, dx, np.ascontiguousarray(U), np.ascontiguousarray(Wx), np.ascontiguousarray(Wy))
    P = oracle.params(gamma=gamma, mu=mu, Pr=Pr)

    def amplitude():  # the right-going wave's rho' + u'/c
        r = st.U[0, 0]
        return abs(np.fft.rfft(r - r.mean() + st.U[1, 0] / r / c)[1]) / nx

    a0 = amplitude()
    while st.t < t_end:
        assert oracle.step2d(P, st, oracle.bcs([0, 0, 0, 0]), 0.5, dt_max=t_end - st.t, viscous_dt=1)[0] == 0
    N = 2 / (gamma - 1)
    return math.log(a0 / amplitude()) / st.t, 0.5 * k * k * (2 * mu * (N - 1) / N + (gamma - 1) * mu / Pr)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_acoustic_damping_is_the_navier_stokes_one(gamma):
    """Sound waves damp at the Navier-Stokes rate of the BGK gas: within 2% at Pr = 1 (32 and 64
    cells per wavelength).  With the Prandtl correction (Pr = 0.72) the damping exceeds it by an
    amount that vanishes with resolution (measured +14-17% at 32 cells, +3-5% at 64)."""
    for nx in (32, 64):
        rate, ns = _acoustic_damping(nx, gamma, 1.0)
        assert rate == pytest.approx(ns, rel=2e-2)
    e32 = _acoustic_damping(32, gamma, 0.72)
    e64 = _acoustic_damping(64, gamma, 0.72)
    excess32, excess64 = e32[0] / e32[1] - 1, e64[0] / e64[1] - 1
    assert 0 < excess64 < 0.06 and excess64 < excess32 / 3
