"""Brute-force velocity-space quadrature used to pin the oracle.

Nothing here calls the oracle.  Moments are integrals of the Maxwellian over (u, v) by
Gauss-Legendre on a truncated range (split at u = 0 for half spaces), with the internal
degrees of freedom integrated through chi-square moments of xi^2 (scipy.stats.chi2).
The interface distribution is built from its definitions in Section 2.2 -- the integral
solution (Eq. integral), the Taylor expansion of f0 (Eq. f0) with the Navier-Stokes
f_G (Eq. ns) and of g (Eq. equli) -- and integrated in time and along the face by
Gauss-Legendre, so the paper's C_1..C_8 and the expanded Eq. dis1 / dis2 are not used.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.stats as st

NV = 40     # velocity nodes per segment
SPAN = 11.0  # half width of the velocity range in standard deviations
RMAX = 3    # highest power of xi^2 carried


def xi_moments(K: float, lam: float):
    """<(xi^2)^r> for r = 0..RMAX, xi^2 = (1/(2 lam)) chi^2_K."""
    s2 = 1.0 / (2.0 * lam)
    return np.array([1.0] + [st.chi2(K).moment(r) * s2 ** r for r in range(1, RMAX + 1)])


def gl(a: float, b: float, n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


class Dist:
    """A Maxwellian with its (u, v) quadrature grid restricted to one u-range."""

    def __init__(self, rho, U, V, lam, K, half=0):
        self.rho, self.U, self.V, self.lam, self.K = rho, U, V, lam, K
        s = 1.0 / math.sqrt(2.0 * lam)
        lo, hi = U - SPAN * s, U + SPAN * s
        if half == 1:
            lo = max(lo, 0.0)
        elif half == 2:
            hi = min(hi, 0.0)
        if half == 0 and lo < 0.0 < hi:
            u1, w1 = gl(lo, 0.0, NV)
            u2, w2 = gl(0.0, hi, NV)
            u, wu = np.concatenate([u1, u2]), np.concatenate([w1, w2])
        elif hi > lo:
            u, wu = gl(lo, hi, 2 * NV)
        else:
            u, wu = np.zeros(1), np.zeros(1)
        v, wv = gl(V - SPAN * s, V + SPAN * s, 2 * NV)
        self.u, self.v = np.meshgrid(u, v, indexing="ij")
        g2 = rho * (lam / math.pi) * np.exp(-lam * ((self.u - U) ** 2 + (self.v - V) ** 2))
        self.w = g2 * wu[:, None] * wv[None, :]
        self.xi = xi_moments(K, lam)

    # a velocity function is an array [RMAX+1, nu, nv] of coefficients of (xi^2)^r
    def const(self, c=1.0):
        f = np.zeros((RMAX + 1,) + self.u.shape)
        f[0] = c
        return f

    def U_(self):
        f = self.const(0.0); f[0] = self.u; return f

    def V_(self):
        f = self.const(0.0); f[0] = self.v; return f

    def psi(self):
        e = self.const(0.0)
        e[0] = 0.5 * (self.u ** 2 + self.v ** 2)
        e[1] = 0.5
        return [self.const(1.0), self.U_(), self.V_(), e]

    def coef(self, X):
        p = self.psi()
        return X[0] * p[0] + X[1] * p[1] + X[2] * p[2] + X[3] * p[3]

    @staticmethod
    def mul(a, b):
        out = np.zeros_like(a)
        for r in range(RMAX + 1):
            for s in range(RMAX + 1 - r):
                out[r + s] += a[r] * b[s]
        return out

    def mom(self, f):
        """int g f dXi (not normalised)."""
        return sum(self.xi[r] * np.sum(self.w * f[r]) for r in range(RMAX + 1))

    def mom4(self, f):
        return np.array([self.mom(self.mul(f, p)) for p in self.psi()])


def prim(w, gamma):
    rho = w[0]
    U, V = w[1] / rho, w[2] / rho
    p = (gamma - 1.0) * (w[3] - 0.5 * rho * (U * U + V * V))
    return rho, U, V, p


def dist_from_cons(w, gamma, half=0):
    K = (4.0 - 2.0 * gamma) / (gamma - 1.0)
    rho, U, V, p = prim(w, gamma)
    return Dist(rho, U, V, rho / (2.0 * p), K, half)


def solve(d: Dist, rhs):
    """a with int g a psi = rhs, a expanded in psi."""
    p = d.psi()
    M = np.array([[d.mom(d.mul(p[a], p[b])) for a in range(4)] for b in range(4)])
    return np.linalg.solve(M, np.asarray(rhs, dtype=np.float64))


def coef_set(d: Dist, dn, dt, dnn, dnt, dtt):
    """The nine coefficient functions of one Maxwellian (system after Eq. dis3)."""
    c = {}
    c["a1"] = solve(d, dn)
    c["a2"] = solve(d, dt)
    c["Axx"] = solve(d, dnn)
    c["Axy"] = solve(d, dnt)
    c["Ayy"] = solve(d, dtt)
    u, v = d.U_(), d.V_()
    M = d.mul
    c["A"] = solve(d, -(d.mom4(M(d.coef(c["a1"]), u)) + d.mom4(M(d.coef(c["a2"]), v))))
    c["Atx"] = solve(d, -(d.mom4(M(d.coef(c["Axx"]), u)) + d.mom4(M(d.coef(c["Axy"]), v))))
    c["Aty"] = solve(d, -(d.mom4(M(d.coef(c["Axy"]), u)) + d.mom4(M(d.coef(c["Ayy"]), v))))
    c["Att"] = solve(d, -(d.mom4(M(d.coef(c["Atx"]), u)) + d.mom4(M(d.coef(c["Aty"]), v))))
    return c


def face_flux(L, R, U0_derivs, gamma, mu, Pr, tau, dtan, dt, ns, nt=24, ntp=24):
    """Time-integrated face-mean flux and Gauss-point values at t = dt.

    L, R: [6][4] face-frame value and derivatives of the two sides; U0_derivs: the
    equilibrium state's (U0, dn, dt, dnn, dnt, dtt).  ns selects the Navier-Stokes f_G.
    Returns (F[4], Wg[2][4], q) with q the time-integrated face-mean heat flux.
    """
    L, R, G = (np.asarray(a, dtype=np.float64) for a in (L, R, U0_derivs))
    g0 = dist_from_cons(G[0], gamma, 0)
    gl_ = dist_from_cons(L[0], gamma, 1)
    gr_ = dist_from_cons(R[0], gamma, 2)
    # the coefficients of each side are fixed by that Maxwellian's full-space moments
    c0 = coef_set(g0, *G[1:])
    cl = coef_set(dist_from_cons(L[0], gamma, 0), *L[1:])
    cr = coef_set(dist_from_cons(R[0], gamma, 0), *R[1:])
    rho0, U0, V0, _ = prim(G[0], gamma)

    def kinetic(d, c, t, y):
        """exp(-t/tau) f0(-u t, y - v t) with f0 the Taylor expansion of f_G."""
        x_, y_ = -d.u * t, y - d.v * t
        C = lambda k: d.coef(c[k])
        u, v = d.U_(), d.V_()
        M = d.mul
        one = d.const(1.0)
        if ns:
            f00 = one - tau * (M(C("a1"), u) + M(C("a2"), v) + C("A"))
            fx = C("a1") - tau * (M(C("Axx"), u) + M(C("Axy"), v) + C("Atx"))
            fy = C("a2") - tau * (M(C("Axy"), u) + M(C("Ayy"), v) + C("Aty"))
        else:
            f00, fx, fy = one, C("a1"), C("a2")
        f = f00 + fx * x_ + fy * y_ + 0.5 * C("Axx") * x_ ** 2 + C("Axy") * x_ * y_ + 0.5 * C("Ayy") * y_ ** 2
        return math.exp(-t / tau) * f

    def hydro(d, c, t, y):
        """(1/tau) int_0^t g(x', y', t') exp(-(t-t')/tau) dt' along x' = -u(t-t'), y' = y - v(t-t')."""
        C = lambda k: d.coef(c[k])
        out = d.const(0.0)
        if t <= 0.0:
            return out
        tp, wp = gl(0.0, t, ntp)
        for s, ws in zip(tp, wp):
            x_, y_ = -d.u * (t - s), y - d.v * (t - s)
            gpoly = (d.const(1.0) + C("a1") * x_ + C("a2") * y_ + C("A") * s
                     + 0.5 * C("Axx") * x_ ** 2 + C("Axy") * x_ * y_ + 0.5 * C("Ayy") * y_ ** 2
                     + 0.5 * C("Att") * s ** 2 + C("Atx") * x_ * s + C("Aty") * y_ * s)
            out += (ws / tau) * math.exp(-(t - s) / tau) * gpoly
        # Eq. dis1 drops tau^2 (1 - exp(-t/tau)) D^2 g (Burnett order) from the second-order
        # weights: remove 2 tau^2 (1 - e) Q(x' = -u, y' - y = -v, t' = -1), Q the quadratic part
        u, v = d.U_(), d.V_()
        M = d.mul
        q2 = (0.5 * M(C("Axx"), M(u, u)) + M(C("Axy"), M(u, v)) + 0.5 * M(C("Ayy"), M(v, v))
              + M(C("Atx"), u) + M(C("Aty"), v) + 0.5 * C("Att"))
        out -= 2.0 * tau * tau * (1.0 - math.exp(-t / tau)) * q2
        return out

    def moments_at(t, y, weight):
        tot = np.zeros(4)
        q = 0.0
        for d, c, part in ((g0, c0, hydro), (gl_, cl, kinetic), (gr_, cr, kinetic)):
            f = part(d, c, t, y)
            if weight == "u":
                tot += d.mom4(d.mul(f, d.U_()))
                cu = d.U_() - U0 * d.const(1.0)
                cv = d.V_() - V0 * d.const(1.0)
                e2 = 0.5 * (d.mul(cu, cu) + d.mul(cv, cv))
                e2[1] += 0.5
                q += d.mom(d.mul(f, d.mul(cu, e2)))
            else:
                tot += d.mom4(f)
        return tot, q

    ts, wts = gl(0.0, dt, nt)
    ys, wys = gl(-0.5 * dtan, 0.5 * dtan, 3)
    F = np.zeros(4)
    q = 0.0
    for t, wt in zip(ts, wts):
        for y, wy in zip(ys, wys):
            m, qq = moments_at(t, y, "u")
            F += wt * wy / dtan * m
            q += wt * wy / dtan * qq
    if Pr != 1.0:
        F[3] += (1.0 / Pr - 1.0) * q
    yg = math.sqrt(3.0) / 6.0 * dtan
    Wg = np.array([moments_at(dt, -yg, "psi")[0], moments_at(dt, yg, "psi")[0]])
    return F, Wg, q
