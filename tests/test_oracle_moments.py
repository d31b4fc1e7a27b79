"""Pins of the oracle's Maxwellian moments and coefficient solves (Section 2.1, 2.2).

Each value is checked against something the oracle does not compute itself: scipy
quadrature of the Gaussian, chi-square moments for the internal degrees of freedom,
the identity half(u>0) + half(u<0) = full, and brute-force velocity quadrature
(tests/bruteforce.py) for the solves of <a> = rhs.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.stats as st

import oracle
import bruteforce as bf

CASES = [(0.3, -0.2, 2.0, 3.0), (-1.1, 0.4, 0.7, 1.0), (0.0, 0.0, 1.0, 3.0), (2.5, -1.5, 4.0, 1.0)]


@pytest.mark.parametrize("U,V,lam,K", CASES)
def test_half_space_moments_sum_to_full(U, V, lam, K):
    full, _, _ = oracle.moments(U, V, lam, K, 0)
    pos, _, _ = oracle.moments(U, V, lam, K, 1)
    neg, _, _ = oracle.moments(U, V, lam, K, 2)
    np.testing.assert_allclose(pos + neg, full, rtol=1e-13, atol=1e-14 * np.abs(full).max())


@pytest.mark.parametrize("U,V,lam,K", CASES)
def test_moments_against_quadrature(U, V, lam, K):
    dens = lambda u, m: math.sqrt(lam / math.pi) * math.exp(-lam * (u - m) ** 2)
    for half, (lo, hi) in ((0, (-np.inf, np.inf)), (1, (0.0, np.inf)), (2, (-np.inf, 0.0))):
        mu, mv, mx = oracle.moments(U, V, lam, K, half)
        for n in range(10):
            ref = si.quad(lambda u: u ** n * dens(u, U), lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            assert mu[n] == pytest.approx(ref, rel=1e-9, abs=1e-13)
        for n in range(10):
            ref = si.quad(lambda v: v ** n * dens(v, V), -np.inf, np.inf, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            assert mv[n] == pytest.approx(ref, rel=1e-9, abs=1e-13)
    s2 = 1.0 / (2.0 * lam)
    assert mx[1] == pytest.approx(st.chi2(K).moment(1) * s2, rel=1e-14)
    assert mx[2] == pytest.approx(st.chi2(K).moment(2) * s2 ** 2, rel=1e-14)


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_moments_reproduce_conservative_variables(gamma):
    """rho <psi> = (rho, rho U, rho V, rho E) with rho E = rho|U|^2/2 + p/(gamma-1) (Section 2.1)."""
    K = (4.0 - 2.0 * gamma) / (gamma - 1.0)
    rho, U, V, p = 0.8, 0.3, -0.7, 1.3
    lam = rho / (2.0 * p)
    mu, mv, mx = oracle.moments(U, V, lam, K, 0)
    E = 0.5 * (mu[2] + mv[2] + mx[1])
    got = rho * np.array([1.0, mu[1], mv[1], E])
    want = np.array([rho, rho * U, rho * V, 0.5 * rho * (U * U + V * V) + p / (gamma - 1.0)])
    np.testing.assert_allclose(got, want, rtol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_coefficient_solve_against_quadrature(seed):
    rng = np.random.default_rng(seed)
    rho, U, V = rng.uniform(0.3, 2.0), rng.uniform(-1, 1), rng.uniform(-1, 1)
    lam, K = rng.uniform(0.3, 3.0), [1.0, 3.0][seed % 2]
    rhs = rng.normal(size=4)
    a = oracle.solve_coef(rho, U, V, lam, K, rhs)
    d = bf.Dist(rho, U, V, lam, K)
    # the defining equation: int g a psi dXi = rhs
    np.testing.assert_allclose(d.mom4(d.coef(a)), rhs, rtol=1e-11, atol=1e-12 * np.abs(rhs).max())


def test_coefficient_solve_basis_round_trip():
    rho, U, V, lam, K = 1.3, 0.2, -0.4, 1.7, 3.0
    d = bf.Dist(rho, U, V, lam, K)
    for k in range(4):
        e = np.zeros(4)
        e[k] = 1.0
        rhs = d.mom4(d.coef(e))
        np.testing.assert_allclose(oracle.solve_coef(rho, U, V, lam, K, rhs), e, atol=1e-11)
