"""Pins of the time coefficients C_1..C_8 (Section 2.2) and their closed-form integrals.

C_k(t) are checked against their definition as time integrals of the BGK solution
(Eq. integral): (1/tau) int_0^t s^m exp(-(t-s)/tau) ds and exp(-t/tau) t^m; the closed
forms of int_0^T C_k(t) dt against 40-digit mpmath quadrature.
"""
import mpmath as mp
import numpy as np
import pytest

import oracle

mp.mp.dps = 40


def _weights(t, tau):
    """Weights of the integral solution (Eq. integral) along x' = -u (t-s), t' = s:
    (1/tau) int_0^t m(s) exp(-(t-s)/tau) ds for m = 1, (t-s), s, (t-s)^2, s^2, (t-s) s."""
    t, tau = mp.mpf(t), mp.mpf(tau)
    I = lambda f: mp.quad(lambda s: f(s) * mp.exp(-(t - s) / tau), [0, t]) / tau
    return {"1": I(lambda s: 1), "r": I(lambda s: t - s), "s": I(lambda s: s),
            "rr": I(lambda s: (t - s) ** 2), "ss": I(lambda s: s ** 2), "rs": I(lambda s: (t - s) * s)}


@pytest.mark.parametrize("t,tau", [(0.3, 0.1), (1.0, 2.0), (0.02, 0.001), (0.5, 0.5)])
def test_C_values_against_the_integral_solution(t, tau):
    """C1, C2, C3 are the exact weights of 1, x' = -u(t-s) and t'; C7, C8 those of the kinetic
    part exp(-t/tau) (1, x = -u t).  The second-order weights C4, C5, C6 of Eq. dis1 are the exact
    ones minus 2 tau^2 (1 - exp(-t/tau)): the paper drops tau^2 D^2 g, a Burnett-order term,
    consistently with the Navier-Stokes truncation of f_G (Eq. ns)."""
    c = oracle.time_coefs(t, tau)
    w = _weights(t, tau)
    e = mp.exp(-mp.mpf(t) / tau)
    drop = 2 * mp.mpf(tau) ** 2 * (1 - e)
    want = {1: w["1"], 2: -w["r"], 3: w["s"], 4: w["rr"] - drop, 5: w["ss"] - drop, 6: -w["rs"] - drop,
            7: e, 8: -t * e, 9: t * e, 10: t * t * e}
    for k, v in want.items():
        assert c[k] == pytest.approx(float(v), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("T,tau", [(0.7, 0.3), (1e-2, 5e-4), (1e-3, 0.02), (2.0, 0.1), (0.05, 0.0025), (1e-3, 0.1)])
def test_time_integrals_against_quadrature(T, tau):
    got = oracle.time_integrals(T, tau)
    for k in range(1, 11):
        f = lambda t, k=k: _fun(k, t, mp.mpf(tau))
        ref = mp.quad(f, [0, mp.mpf(T)])
        # the closed forms lose about 1/x^3 of their digits at x = T/tau << 1 (cancellation);
        # x >= 0.01 covers every workload here
        assert got[k] == pytest.approx(float(ref), rel=1e-8, abs=1e-15 * T ** 3)


def _fun(k, t, tau):
    e = mp.exp(-t / tau)
    return [None, 1 - e, (t + tau) * e - tau, t - tau + tau * e, -(t * t + 2 * t * tau) * e, t * t - 2 * t * tau,
            -t * tau * (1 + e), e, -t * e, t * e, t * t * e][k]


def test_collision_free_limit():
    """tau = 0: the equilibrium part alone, C1 = 1, C3 = t, C5 = t^2, the rest 0."""
    T = 0.3
    c = oracle.time_coefs(T, 0.0)
    assert list(c[1:9]) == [1.0, 0.0, T, 0.0, T * T, 0.0, 0.0, 0.0]
    ci = oracle.time_integrals(T, 0.0)
    np.testing.assert_allclose(ci[1:11], [T, 0, T * T / 2, 0, T ** 3 / 3, 0, 0, 0, 0, 0], atol=1e-17)


def test_smooth_cancellation_identities():
    """The identities behind Eq. dis3: C1 + C7 = 1, C2 + C8 - tau C7 = -tau, C3 - tau C7 = t - tau."""
    for t, tau in [(0.1, 0.03), (1.0, 5.0), (2.0, 0.01)]:
        c = oracle.time_coefs(t, tau)
        assert c[1] + c[7] == pytest.approx(1.0, abs=1e-15)
        assert c[2] + c[8] - tau * c[7] == pytest.approx(-tau, rel=1e-13)
        assert c[3] - tau * c[7] == pytest.approx(t - tau, rel=1e-13, abs=1e-15)
