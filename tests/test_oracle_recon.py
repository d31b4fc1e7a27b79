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
