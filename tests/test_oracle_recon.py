"""Pins of the oracle's compact reconstruction (Section 3) and boundary images.

A quadratic is reproduced exactly by every stencil (Eq. over-sys, the limiter of
Eq. limiter and the central stencil), so the reconstruction must return its
coefficients; a jump must switch the weights of Eq. average to the limited stencil.
The wall images are checked by finite differences of their pointwise definition, and by
the symmetry of the mirrored interface (no mass flux through a wall).
"""
import math

import numpy as np
import pytest

import oracle

G = math.sqrt(3.0) / 6.0


def _cons(rho, u, v, p, gamma):
    return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def _quadratic_cell(seed, dx, dy, gamma=1.4):
    rng = np.random.default_rng(seed)
    base = _cons(1.0, 0.2, -0.1, 1.0, gamma)
    a = np.zeros((4, 6))
    a[:, 0] = base
    a[:, 1:] = rng.normal(scale=0.3, size=(4, 5))
    # Q(x, y) = Ubar + a2 x + a3 y + a4 (x^2 - dx^2/12)/2 + a5 (y^2 - dy^2/12)/2 + a6 x y
    Q = lambda x, y: (a[:, 0] + a[:, 1] * x + a[:, 2] * y + a[:, 3] * 0.5 * (x * x - dx * dx / 12)
                      + a[:, 4] * 0.5 * (y * y - dy * dy / 12) + a[:, 5] * x * y)
    avg = lambda cx, cy: (a[:, 0] + a[:, 1] * cx + a[:, 2] * cy + a[:, 3] * 0.5 * cx * cx
                          + a[:, 4] * 0.5 * cy * cy + a[:, 5] * cx * cy)
    nb = np.array([avg(0, 0), avg(dx, 0), avg(-dx, 0), avg(0, dy), avg(0, -dy)])
    fx = np.array([Q(dx / 2, -G * dy), Q(dx / 2, G * dy), Q(-dx / 2, -G * dy), Q(-dx / 2, G * dy)])
    fy = np.array([Q(-G * dx, dy / 2), Q(G * dx, dy / 2), Q(-G * dx, -dy / 2), Q(G * dx, -dy / 2)])
    return a, nb, fx, fy


@pytest.mark.parametrize("seed", range(6))
def test_reconstruction_exact_for_quadratics(seed):
    dx, dy = 0.05, 0.03 + 0.01 * seed
    a, nb, fx, fy = _quadratic_cell(seed, dx, dy)
    got = oracle.recon_cell(oracle.params(), nb, fx, fy, dx, dy)
    np.testing.assert_allclose(got, a, rtol=1e-9, atol=1e-9)


def test_reconstruction_1d_exact_for_quadratics():
    rng = np.random.default_rng(3)
    dx = 0.04
    a = np.array([[1.0, 0.3, -2.0], [0.2, -0.5, 1.0], [2.6, 0.1, 0.4]])
    Q = lambda x: a[:, 0] + a[:, 1] * x + a[:, 2] * 0.5 * (x * x - dx * dx / 12)
    avg = lambda c: a[:, 0] + a[:, 1] * c + a[:, 2] * 0.5 * c * c
    nb = np.array([avg(0.0), avg(-dx), avg(dx)])
    fw = np.array([Q(-dx / 2), Q(dx / 2)])
    P = oracle.params()
    out = np.zeros((3, 3))
    import ctypes
    oracle.lib().orc1d_recon_cell(ctypes.byref(P), oracle._p(np.ascontiguousarray(nb)),
                                  oracle._p(np.ascontiguousarray(fw)), dx, oracle._p(out))
    np.testing.assert_allclose(out, a, rtol=1e-10, atol=1e-10)
    del rng


def test_reconstruction_at_a_jump_uses_the_limited_stencil():
    """Across a density jump the central slope is O(jump/dx) but the one-sided pair disagrees in
    sign of curvature; the weights must suppress the central polynomial (Eq. average)."""
    dx = dy = 0.02
    lo, hi = _cons(0.2, 0, 0, 0.3, 1.4), _cons(1.0, 0, 0, 1.0, 1.4)
    nb = np.array([lo, hi, lo, lo, lo])  # the east neighbour sits across a jump
    fx = np.array([0.5 * (lo + hi)] * 2 + [lo, lo])
    fy = np.array([lo, lo, lo, lo])
    got = oracle.recon_cell(oracle.params(), nb, fx, fy, dx, dy)
    central_slope = (hi[0] - lo[0]) / (2 * dx)
    assert abs(got[0, 1]) < 1e-3 * central_slope
    # the central curvature (hi - lo)/dx^2 enters only with the small weight omega_2, about
    # (I(U1) / I(U2))^2 = (C dx dy / (jump^2 ...))^2 ~ 1e-4 here
    assert np.all(np.abs(got[:, 2:]) < 1e-3 * (hi[0] - lo[0]) / dx ** 2)


def test_positivity_fallback():
    """A cell whose polynomial would give negative density at a face centre is made constant."""
    dx = dy = 0.1
    c = _cons(0.05, 0, 0, 0.05, 1.4)
    big = _cons(3.0, 0, 0, 3.0, 1.4)
    nb = np.array([c, big, c, c, c])
    fx = np.array([big, big, c, c])  # a steep rise on the east face only
    fy = np.array([c, c, c, c])
    got = oracle.recon_cell(oracle.params(weno_C=1e6), nb, fx, fy, dx, dy)
    # a2 > 0 with a4 curvature would push the west face below zero; either the fit stays
    # positive at all four face centres or it is the constant
    x = np.array([dx / 2, -dx / 2, 0, 0])
    y = np.array([0, 0, dy / 2, -dy / 2])
    vals = got[0, 0] + got[0, 1] * x + got[0, 2] * y + got[0, 3] * 0.5 * (x * x - dx * dx / 12) \
        + got[0, 4] * 0.5 * (y * y - dy * dy / 12) + got[0, 5] * x * y
    assert np.all(vals > 0)


# ---------------- boundary images ----------------

def _prim_image(w, gamma, kind, uwt, Tw):
    """Pointwise wall map in primitive variables: rho' = rho, u_n' = -u_n,
    slip: u_t' = u_t, T' = T; no-slip isothermal: u_t' = 2 u_wt - u_t, T' = 2 T_w - T;
    no-slip adiabatic: u_t' = 2 u_wt - u_t, T' = T."""
    rho, un, ut = w[0], w[1] / w[0], w[2] / w[0]
    T = (gamma - 1) * (w[3] / rho - 0.5 * (un * un + ut * ut))
    if kind == oracle.BC_SLIPWALL:
        return _cons(rho, -un, ut, rho * T, gamma)
    if kind == oracle.BC_NOSLIP_ADIABATIC:
        return _cons(rho, -un, 2 * uwt - ut, rho * T, gamma)
    return _cons(rho, -un, 2 * uwt - ut, rho * (2 * Tw - T), gamma)


@pytest.mark.parametrize("kind", [oracle.BC_SLIPWALL, oracle.BC_NOSLIP_ISOTHERMAL, oracle.BC_NOSLIP_ADIABATIC])
def test_wall_image_derivatives(kind):
    gamma, uwt, Tw = 1.4, 0.15, 0.7
    rng = np.random.default_rng(5)
    S = np.zeros((6, 4))
    S[0] = _cons(1.1, 0.2, -0.3, 0.8, gamma)
    S[1:] = rng.normal(scale=0.3, size=(5, 4))
    P_in = lambda n, t: S[0] + S[1] * n + S[2] * t + 0.5 * S[3] * n * n + S[4] * n * t + 0.5 * S[5] * t * t
    Gf = lambda n, t: _prim_image(P_in(-n, t), gamma, kind, uwt, Tw)
    h = 1e-3
    want = np.array([
        Gf(0, 0),
        (Gf(h, 0) - Gf(-h, 0)) / (2 * h),
        (Gf(0, h) - Gf(0, -h)) / (2 * h),
        (Gf(h, 0) - 2 * Gf(0, 0) + Gf(-h, 0)) / h ** 2,
        (Gf(h, h) - Gf(h, -h) - Gf(-h, h) + Gf(-h, -h)) / (4 * h * h),
        (Gf(0, h) - 2 * Gf(0, 0) + Gf(0, -h)) / h ** 2,
    ])
    got = oracle.bc_image(oracle.params(gamma=gamma), kind, uwt, Tw, S)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("mu", [0.0, 2e-3])
def test_slip_wall_face_is_impermeable(mu):
    """A face between a state and its slip-wall mirror (with mirrored cell averages) carries no
    mass, tangential momentum or energy flux: the interface distribution is symmetric in u."""
    gamma = 1.4
    rng = np.random.default_rng(8)
    S = np.zeros((6, 4))
    S[0] = _cons(1.0, 0.3, -0.2, 0.9, gamma)
    S[1:] = rng.normal(scale=0.3, size=(5, 4))
    P = oracle.params(gamma=gamma, mu=mu, Pr=0.72)
    img = oracle.bc_image(P, oracle.BC_SLIPWALL, 0.0, 1.0, S)
    avg = np.zeros((2, 3, 4))
    for k in range(3):
        avg[1, k] = _cons(1.0 + 0.05 * k, 0.3, -0.2 + 0.02 * k, 0.9, gamma)
        avg[0, k] = _prim_image(avg[1, k], gamma, oracle.BC_SLIPWALL, 0.0, 1.0)
    F, Wg, _ = oracle.face(P, img, S, avg, 0.05, 0.05, 0.01)
    scale = abs(F[1])
    assert abs(F[0]) < 1e-13 * scale and abs(F[2]) < 1e-13 * scale and abs(F[3]) < 1e-13 * scale
    assert np.all(np.abs(Wg[:, 1]) < 1e-13)


# ---------------- the smallest-|a6| choice and the nonlinear weights ----------------
#
# Eq. over-sys solves each one-sided stencil in the least-squares sense.  Its cross
# coefficient a6 enters only the four Gauss-point conditions of the stencil's two faces
# (the neighbour averages do not see x y), so with Ubar, a2..a5 held, a6^k is the
# least-squares solution of those four conditions.  The tests below compute it that way,
# from the point coordinates alone, and never from the oracle's closed form.

_STENCILS = ((1, 1), (-1, 1), (-1, -1), (1, -1))  # the order of Section 3.2's stencils 1..4


def _gauss_points(sx, sy, dx, dy):
    """(x, y, slot) of the four Gauss points of stencil (sx, sy): its x-face x = sx dx/2 at
    y = -/+ sqrt(3)/6 dy (slots of fx), and its y-face y = sy dy/2 at x = -/+ sqrt(3)/6 dx
    (slots of fy)."""
    ex = 0 if sx > 0 else 2
    ey = 0 if sy > 0 else 2
    return ([(sx * dx / 2, -G * dy, ("x", ex)), (sx * dx / 2, G * dy, ("x", ex + 1))] +
            [(-G * dx, sy * dy / 2, ("y", ey)), (G * dx, sy * dy / 2, ("y", ey + 1))])


def _lstsq_cross(coef, fx, fy, dx, dy, sx, sy):
    """a6 of one-sided stencil (sx, sy) for one variable: least squares over its four
    Gauss-point conditions, coef = (Ubar, a2, a3, a4, a5) held."""
    c0, a2, a3, a4, a5 = coef
    rows, rhs = [], []
    for x, y, (face, k) in _gauss_points(sx, sy, dx, dy):
        val = fx[k] if face == "x" else fy[k]
        rows.append([x * y])
        rhs.append(val - (c0 + a2 * x + a3 * y + a4 * 0.5 * (x * x - dx * dx / 12)
                          + a5 * 0.5 * (y * y - dy * dy / 12)))
    return float(np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0][0])


def _cell_with_face_differences(seed, dx, dy, z):
    """A quadratic cell (averages and Gauss-point values) whose face Gauss-point pairs are
    then pulled apart: the y+ (x+) value of face f rises by z[f] and the y- (x-) value falls by
    z[f], f = east, west, north, south, per variable.  The face means, hence the one-sided
    a2..a5 (and the central a2..a5), stay those of the quadratic."""
    a, nb, fx, fy = _quadratic_cell(seed, dx, dy)
    fx, fy = fx.copy(), fy.copy()
    ze, zw, zn, zs = (np.asarray(z[k], dtype=float) for k in range(4))
    fx[0] -= ze; fx[1] += ze
    fx[2] -= zw; fx[3] += zw
    fy[0] -= zn; fy[1] += zn
    fy[2] -= zs; fy[3] += zs
    return a, nb, fx, fy


# weights that keep only the one-sided polynomial: I(U1) = C dx dy ~ 1e-33 against
# I(U2) ~ 1e-4, so omega_2 ~ 1e-58 and the output is the one-sided polynomial itself
_ONE_SIDED = dict(weno_eps=0.0, weno_C=1e-30)


def _expected_choice(a, fx, fy, dx, dy, v):
    cands = [_lstsq_cross(a[v, :5], fx[:, v], fy[:, v], dx, dy, sx, sy) for sx, sy in _STENCILS]
    return cands


def test_cross_derivative_keeps_the_smallest_stencil():
    """Section 3.2: of the four one-sided cross derivatives the one with the smallest absolute
    value is kept.  Variable v of the cell is built so that stencil v is the smallest, with
    a clear margin, so every position of the order is exercised and a reversed comparison,
    a wrong sign in any stencil or the wrong face of a stencil changes the result."""
    dx, dy = 0.04, 0.03
    rng = np.random.default_rng(17)
    z = np.zeros((4, 4))
    a = None
    for v in range(4):
        for _ in range(1000):
            z[:, v] = rng.normal(scale=2e-4, size=4)
            a, nb, fx, fy = _cell_with_face_differences(11, dx, dy, z)
            c = np.abs(_expected_choice(a, fx, fy, dx, dy, v))
            order = np.argsort(c)
            if order[0] == v and c[order[1]] > 1.3 * c[order[0]]:
                break
        else:
            raise AssertionError("no draw makes stencil %d the smallest" % v)
    a, nb, fx, fy = _cell_with_face_differences(11, dx, dy, z)
    got = oracle.recon_cell(oracle.params(**_ONE_SIDED), nb, fx, fy, dx, dy)
    # the face means are untouched: the limited one-sided a2..a5 are the quadratic's
    np.testing.assert_allclose(got[:, :5], a[:, :5], rtol=1e-9, atol=1e-9)
    for v in range(4):
        cands = _expected_choice(a, fx, fy, dx, dy, v)
        assert int(np.argmin(np.abs(cands))) == v
        assert got[v, 5] == pytest.approx(cands[v], rel=1e-9, abs=1e-9), (v, cands)
        # and it is not any of the other three
        for k in range(4):
            if k != v:
                assert abs(got[v, 5] - cands[k]) > 1e-3 * abs(cands[k] - cands[v])


# (z_east, z_west, z_north, z_south) in units of tau, and the stencil whose a6 is kept:
# in each case two candidates tie at +-k tau (opposite signs) and the other two are
# 9 k tau and 11 k tau, with k = 2 sqrt(3) / (dx dy); the earlier stencil of the tie wins
_TIES = [
    ((1, 1, 0, -10), 0),   # (+,+) = k tau, (-,+) = -k tau
    ((10, 0, 1, 1), 1),    # (-,+) = k tau, (-,-) = -k tau
    ((1, 1, 10, 0), 2),    # (-,-) = -k tau, (+,-) = k tau
    ((0, -10, 1, 1), 0),   # (+,+) = k tau, (+,-) = -k tau
]


@pytest.mark.parametrize("zs,keep", _TIES)
def test_cross_derivative_tie_keeps_the_earlier_stencil(zs, keep):
    """The paper gives no tie rule; the reading keeps the first stencil of the order
    (+,+), (-,+), (-,-), (+,-).  Exact ties of opposite sign are built from the face
    differences alone (quadratic cross term zero), for each adjacent pair of the order."""
    dx, dy = 0.05, 0.04
    tau = 3e-5
    z = np.array([[zz * tau] * 4 for zz in zs])
    a, nb, fx, fy = _cell_with_face_differences(4, dx, dy, z)
    a6 = a[:, 5].copy()
    # remove the quadratic's own cross term so that the two tied candidates are exactly +-k tau
    for k in range(2):
        fx[k] -= a6 * (dx / 2) * (-G * dy if k == 0 else G * dy)
        fx[2 + k] -= a6 * (-dx / 2) * (-G * dy if k == 0 else G * dy)
        fy[k] -= a6 * (-G * dx if k == 0 else G * dx) * (dy / 2)
        fy[2 + k] -= a6 * (-G * dx if k == 0 else G * dx) * (-dy / 2)
    kk = 2 * math.sqrt(3.0) / (dx * dy)
    got = oracle.recon_cell(oracle.params(**_ONE_SIDED), nb, fx, fy, dx, dy)
    for v in range(4):
        cands = _expected_choice(a, fx, fy, dx, dy, v)
        mags = sorted(abs(c) for c in cands)
        assert mags[0] == pytest.approx(kk * tau, rel=1e-9) and mags[1] == pytest.approx(kk * tau, rel=1e-9)
        assert mags[2] > 8 * kk * tau
        assert got[v, 5] == pytest.approx(cands[keep], rel=1e-7), (v, cands, keep)


def _indicator_by_quadrature(q, dx, dy):
    """I(U) = dx^2 <Ux^2> + dy^2 <Uy^2> + dx^4 Uxx^2 + dx^2 dy^2 Uxy^2 + dy^4 Uyy^2 for
    U = q0 + q1 x + q2 y + q3 wx + q4 wy + q5 x y, with the cell means <.> taken by a 3 x 3
    Gauss-Legendre rule (exact for these quadratics)."""
    t, w = np.polynomial.legendre.leggauss(3)
    X, Y = np.meshgrid(t * dx / 2, t * dy / 2, indexing="ij")
    W = np.outer(w, w) / 4.0
    ux = q[1] + q[3] * X + q[5] * Y
    uy = q[2] + q[4] * Y + q[5] * X
    return (dx * dx * np.sum(W * ux * ux) + dy * dy * np.sum(W * uy * uy) + dx ** 4 * q[3] ** 2
            + dx * dx * dy * dy * q[5] ** 2 + dy ** 4 * q[4] ** 2)


@pytest.mark.parametrize("eps_rel", [0.0, 1.0])
def test_nonlinear_weights_follow_the_inverse_square(eps_rel):
    """Eq. average: omega_i = alpha_i / sum alpha, alpha_i = 1 / (eps + I(U_i))^2, with
    I(U_1) = C dx dy.  The cell is a quadratic Q whose face Gauss values are all shifted
    by a constant per face: the central polynomial (averages and face differences) stays Q,
    the one-sided one does not.  Every output coefficient is then
    Q_k + omega_1(C) (one-sided_k - Q_k), with the one-sided part independent of C, so for
    three values of C the ratio of output differences equals that of omega_1 alone -- which
    fixes the exponent 2 and the place of eps, given I(Q) by quadrature."""
    dx, dy = 0.05, 0.035
    a, nb, fx, fy = _quadratic_cell(21, dx, dy)
    shift = np.array([[2e-3, -1e-3, 5e-4, 1.5e-3], [-8e-4, 1.2e-3, -2e-3, 7e-4],
                      [1e-3, 6e-4, -1.1e-3, -9e-4], [-1.4e-3, -5e-4, 9e-4, 1.6e-3]])  # [face][var]
    fx = fx.copy(); fy = fy.copy()
    fx[0] += shift[0]; fx[1] += shift[0]
    fx[2] += shift[1]; fx[3] += shift[1]
    fy[0] += shift[2]; fy[1] += shift[2]
    fy[2] += shift[3]; fy[3] += shift[3]
    A = dx * dy
    checked = 0
    for v in range(4):
        I2 = _indicator_by_quadrature(a[v], dx, dy)
        eps = eps_rel * I2
        Cs = [0.3 * I2 / A, I2 / A, 3.0 * I2 / A]
        outs = []
        for C in Cs:
            P = oracle.params(weno_eps=eps, weno_C=C)
            outs.append(oracle.recon_cell(P, nb, fx, fy, dx, dy)[v])
        w1 = [(eps + I2) ** 2 / ((eps + C * A) ** 2 + (eps + I2) ** 2) for C in Cs]
        want = (w1[0] - w1[1]) / (w1[1] - w1[2])
        for k in range(1, 6):
            d01, d12 = outs[0][k] - outs[1][k], outs[1][k] - outs[2][k]
            if abs(d12) < 1e-6 * max(1.0, abs(a[v, k])):
                continue  # this coefficient's one-sided value equals the central one
            assert d01 / d12 == pytest.approx(want, rel=1e-7), (v, k)
            # and the output lies on the segment at omega_1 from the central value Q_k
            one_sided = a[v, k] + (outs[1][k] - a[v, k]) / w1[1]
            assert outs[0][k] == pytest.approx(a[v, k] + w1[0] * (one_sided - a[v, k]), rel=1e-8, abs=1e-10)
            checked += 1
    assert checked >= 8
