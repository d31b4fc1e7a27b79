"""Pins of the oracle's interface evolution (Section 2.2) against brute force.

The oracle assembles the flux from the expanded Eq. dis1 / dis2 with closed-form
time integrals and moment tables; tests/bruteforce.py integrates the integral solution
(Eq. integral) with the Taylor expansions of f0 and g numerically in u, v, t and along the
face.  Agreement to ~1e-10 catches a dropped term, a wrong sign or index, a transposed
operand, a wrong y-average or a wrong time integral anywhere in the assembly.
"""
import math

import numpy as np
import pytest

import oracle
import bruteforce as bf


def _cons(rho, u, v, p, gamma):
    return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def random_face(seed, gamma):
    """Left/right face-frame states with derivatives and six nearby cell averages."""
    rng = np.random.default_rng(seed)
    base = (rng.uniform(0.6, 1.4), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.6, 1.4))
    def side():
        r, u, v, p = base
        w = np.zeros((6, 4))
        w[0] = _cons(r * rng.uniform(0.8, 1.2), u + rng.uniform(-0.2, 0.2), v + rng.uniform(-0.2, 0.2),
                     p * rng.uniform(0.8, 1.2), gamma)
        w[1:] = rng.normal(scale=0.4, size=(5, 4))
        return w
    L, R = side(), side()
    avg = np.zeros((2, 3, 4))
    for m in range(2):
        for n in range(3):
            r, u, v, p = base
            avg[m, n] = _cons(r * rng.uniform(0.9, 1.1), u + rng.uniform(-0.1, 0.1), v + rng.uniform(-0.1, 0.1),
                              p * rng.uniform(0.9, 1.1), gamma)
    return L, R, avg


def equilibrium_state(dbg):
    """(U0, d/dn, d/dt, d2/dn2, d2/dndt, d2/dt2) of the equilibrium polynomial from the oracle's b2..b6."""
    U0 = dbg[0:4]
    b = {s: dbg[5 + (s - 2) * 4: 9 + (s - 2) * 4] for s in range(2, 7)}
    return np.array([U0, b[2], b[3], b[4], b[6], b[5]])


CASES = [  # (seed, gamma, mu, Pr, dn, dtan, dt)
    (0, 1.4, 0.0, 1.0, 0.05, 0.05, 0.01),
    (1, 5.0 / 3.0, 0.0, 1.0, 0.04, 0.07, 0.008),
    (2, 1.4, 4e-3, 1.0, 0.05, 0.05, 0.01),
    (3, 1.4, 4e-3, 0.72, 0.03, 0.06, 0.006),
    (4, 5.0 / 3.0, 1e-2, 0.72, 0.05, 0.05, 0.01),
]


@pytest.mark.parametrize("seed,gamma,mu,Pr,dn,dtan,dt", CASES)
def test_face_against_brute_force(seed, gamma, mu, Pr, dn, dtan, dt):
    P = oracle.params(gamma=gamma, mu=mu, Pr=Pr)
    L, R, avg = random_face(seed, gamma)
    F, Wg, dbg = oracle.face(P, L, R, avg, dn, dtan, dt)
    # Eq. compatibility2 by quadrature
    dl, dr = bf.dist_from_cons(L[0], gamma, 1), bf.dist_from_cons(R[0], gamma, 2)
    U0 = dl.mom4(dl.const(1.0)) + dr.mom4(dr.const(1.0))
    np.testing.assert_allclose(dbg[0:4], U0, rtol=1e-12)
    tau = dbg[4]
    G = equilibrium_state(dbg)
    Fb, Wb, qb = bf.face_flux(L, R, G, gamma, mu, Pr, tau, dtan, dt, ns=mu > 0)
    scale = np.abs(Fb).max()
    np.testing.assert_allclose(F, Fb, rtol=1e-10, atol=1e-11 * scale)
    np.testing.assert_allclose(Wg, Wb, rtol=1e-10, atol=1e-11 * np.abs(Wb).max())
    if Pr != 1.0:
        assert dbg[25] == pytest.approx(qb, rel=1e-9, abs=1e-12 * scale)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_collision_time(gamma):
    """Section 4: inviscid tau = eps dt + C |pl-pr|/(pl+pr) dt; viscous tau = mu/p0 + |...| dt."""
    L, R, avg = random_face(7, gamma)
    dt = 0.01
    pl = bf.prim(L[0], gamma)[3]
    pr = bf.prim(R[0], gamma)[3]
    jump = abs(pl - pr) / (pl + pr) * dt
    _, _, dbg = oracle.face(oracle.params(gamma=gamma), L, R, avg, 0.05, 0.05, dt)
    assert dbg[4] == pytest.approx(0.05 * dt + jump, rel=1e-14)
    _, _, dbg = oracle.face(oracle.params(gamma=gamma, mu=2e-3), L, R, avg, 0.05, 0.05, dt)
    p0 = bf.prim(dbg[0:4], gamma)[3]
    assert dbg[4] == pytest.approx(2e-3 / p0 + jump, rel=1e-14)


def _quadratic_face(seed, gamma, dn, dtan):
    """A quadratic field Q(n, t) for every variable: the face-centre value/derivatives, and
    its exact averages over the six cells (m = 0, 1; k = -1, 0, 1) around the face."""
    rng = np.random.default_rng(seed)
    base = _cons(1.0, 0.3, -0.2, 1.0, gamma)
    c = rng.normal(scale=0.2, size=(6, 4))  # value offset, Qn, Qt, Qnn, Qnt, Qtt
    S = np.zeros((6, 4))
    S[0] = base + 0.05 * c[0]
    S[1:] = c[1:]
    avg = np.zeros((2, 3, 4))
    for m in range(2):
        nc = (m - 0.5) * dn
        for k in range(3):
            tc = (k - 1) * dtan
            # cell mean of Q: value + Qn nc + Qt tc + Qnn (nc^2 + dn^2/12)/2 + Qnt nc tc + Qtt (tc^2 + dtan^2/12)/2
            avg[m, k] = (S[0] + S[1] * nc + S[2] * tc + 0.5 * S[3] * (nc * nc + dn * dn / 12)
                         + S[4] * nc * tc + 0.5 * S[5] * (tc * tc + dtan * dtan / 12))
    return S, avg


@pytest.mark.parametrize("seed", range(3))
def test_equilibrium_polynomial_exact_for_quadratics(seed):
    """Section 3.3: the six-average fit with U0 reproduces any quadratic exactly."""
    gamma, dn, dtan = 1.4, 0.05, 0.08
    S, avg = _quadratic_face(seed, gamma, dn, dtan)
    _, _, dbg = oracle.face(oracle.params(gamma=gamma), S, S, avg, dn, dtan, 0.01)
    np.testing.assert_allclose(dbg[0:4], S[0], rtol=1e-13)  # equal sides: U0 = the common value
    G = equilibrium_state(dbg)
    np.testing.assert_allclose(G[1:], S[1:], rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("mu", [3e-3, 1e-2])
def test_smooth_reduction_eq_dis3(mu):
    """Section 2.2: with g_l = g_r = g0 and equal slopes the interface distribution is Eq. dis3.

    Here dis3 is integrated by brute force directly (no C_k, no kinetic part), and must equal
    the oracle's full kinetic + equilibrium assembly (all exp(-t/tau) terms cancel)."""
    gamma, dn, dtan, dt = 1.4, 0.05, 0.05, 0.01
    S, avg = _quadratic_face(11, gamma, dn, dtan)
    P = oracle.params(gamma=gamma, mu=mu)
    F, Wg, dbg = oracle.face(P, S, S, avg, dn, dtan, dt)
    tau = dbg[4]
    d = bf.dist_from_cons(S[0], gamma, 0)
    c = bf.coef_set(d, *S[1:])
    C = lambda k: d.coef(c[k])
    M = d.mul
    u, v, one = d.U_(), d.V_(), d.const(1.0)

    def f_dis3(t, y):
        return (one - tau * (M(C("a1"), u) + M(C("a2"), v) + C("A"))
                + (C("a2") - tau * (M(C("Axy"), u) + M(C("Ayy"), v) + C("Aty"))) * y
                + (C("A") - tau * (M(C("Atx"), u) + M(C("Aty"), v) + C("Att"))) * t
                + 0.5 * C("Ayy") * y * y + C("Aty") * y * t + 0.5 * C("Att") * t * t)

    ts, wt = bf.gl(0.0, dt, 6)
    ys, wy = bf.gl(-dtan / 2, dtan / 2, 3)
    Fd = sum(a * b / dtan * d.mom4(M(f_dis3(t, y), u)) for t, a in zip(ts, wt) for y, b in zip(ys, wy))
    np.testing.assert_allclose(F, Fd, rtol=1e-11, atol=1e-12 * np.abs(Fd).max())
    yg = math.sqrt(3) / 6 * dtan
    for g, y in enumerate((-yg, yg)):
        np.testing.assert_allclose(Wg[g], d.mom4(f_dis3(dt, y)), rtol=1e-11)


def test_uniform_state_flux_is_euler_flux():
    """A uniform state (no gradients) gives the exact Euler flux dt (rho U, rho U^2 + p, rho U V, U(rho E + p))."""
    gamma = 1.4
    rho, U, V, p = 0.9, 0.35, -0.6, 1.2
    w = _cons(rho, U, V, p, gamma)
    S = np.zeros((6, 4))
    S[0] = w
    avg = np.broadcast_to(w, (2, 3, 4)).copy()
    dt = 0.013
    for mu in (0.0, 1e-3):
        F, Wg, _ = oracle.face(oracle.params(gamma=gamma, mu=mu, Pr=0.72), S, S, avg, 0.05, 0.05, dt)
        want = dt * np.array([rho * U, rho * U * U + p, rho * U * V, U * (w[3] + p)])
        np.testing.assert_allclose(F, want, rtol=1e-13)
        np.testing.assert_allclose(Wg, np.array([w, w]), rtol=1e-13)


def test_collisionless_face_against_brute_force():
    """The evolution of the positivity fallback: free transport of the two constant states
    (the tau -> infinity limit of Eq. integral), f = f0 -- flux dt int u psi f0 and point values
    int psi f0 by brute-force half-space quadrature."""
    gamma = 1.4
    L, R, _ = random_face(21, gamma)
    P = oracle.params(gamma=gamma, mu=2e-3, Pr=0.72)
    dt = 0.01
    F, Wg, dbg = oracle.face_first_order(P, L, R, 0.05, 0.05, dt)
    dl, dr = bf.dist_from_cons(L[0], gamma, 1), bf.dist_from_cons(R[0], gamma, 2)
    Fb = dt * (dl.mom4(dl.U_()) + dr.mom4(dr.U_()))
    Wb = dl.mom4(dl.const(1.0)) + dr.mom4(dr.const(1.0))
    np.testing.assert_allclose(F, Fb, rtol=1e-12, atol=1e-13 * np.abs(Fb).max())
    np.testing.assert_allclose(Wg, np.array([Wb, Wb]), rtol=1e-12)
