"""Exact solution of the 1D Euler Riemann problem for an ideal gas (the standard
construction: the star-region pressure is the root of f_L(p) + f_R(p) + u_R - u_L = 0, with
f_K the shock (Rankine-Hugoniot) or rarefaction (isentropic) relation of side K; the
solution is self-similar in x/t).  Test infrastructure for the Sod tube (Section 4.2)."""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, ck, g):
    """f_K(p) and its derivative for the state (rho, pk) with sound speed ck."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk  # rarefaction
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * ck / (g - 1.0) * (r ** e - 1.0), 1.0 / (rho * ck) * r ** (-(g + 1.0) / (2.0 * g))


def star_state(L, R, g=1.4):
    """(p*, u*) for primitive states L = (rho, u, p), R = (rho, u, p)."""
    rl, ul, pl = L
    rr, ur, pr = R
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))  # linearised guess
    for _ in range(100):
        fl, dl = _f(p, rl, pl, cl, g)
        fr, dr = _f(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-14 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(L, R, s, g=1.4):
    """Primitive state (rho, u, p) at x/t = s; the initial discontinuity is at s = 0."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, g)
    if s <= us:  # left of the contact
        rho, u, p, c = rl, ul, pl, math.sqrt(g * pl / rl)
        if ps > pl:  # left shock
            sh = u - c * math.sqrt((g + 1.0) / (2.0 * g) * ps / p + (g - 1.0) / (2.0 * g))
            if s < sh:
                return rho, u, p
            r = (ps / p + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * ps / p + 1.0)
            return rho * r, us, ps
        head = u - c  # left rarefaction
        cs = c * (ps / p) ** ((g - 1.0) / (2.0 * g))
        tail = us - cs
        if s < head:
            return rho, u, p
        if s > tail:
            return rho * (ps / p) ** (1.0 / g), us, ps
        k = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * c) * (u - s)
        return rho * k ** (2.0 / (g - 1.0)), 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * u + s), p * k ** (2.0 * g / (g - 1.0))
    rho, u, p, c = rr, ur, pr, math.sqrt(g * pr / rr)
    if ps > pr:  # right shock
        sh = u + c * math.sqrt((g + 1.0) / (2.0 * g) * ps / p + (g - 1.0) / (2.0 * g))
        if s > sh:
            return rho, u, p
        r = (ps / p + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * ps / p + 1.0)
        return rho * r, us, ps
    head = u + c  # right rarefaction
    cs = c * (ps / p) ** ((g - 1.0) / (2.0 * g))
    tail = us + cs
    if s > head:
        return rho, u, p
    if s < tail:
        return rho * (ps / p) ** (1.0 / g), us, ps
    k = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * c) * (u - s)
    return rho * k ** (2.0 / (g - 1.0)), 2.0 / (g + 1.0) * (-c + 0.5 * (g - 1.0) * u + s), p * k ** (2.0 * g / (g - 1.0))


def cell_average_density(L, R, x0, t, edges, g=1.4, sub=16):
    """Cell averages of the exact density on the cells [edges[i], edges[i+1]] (midpoint rule on
    `sub` sub-intervals per cell)."""
    out = np.zeros(len(edges) - 1)
    for i in range(len(edges) - 1):
        xs = edges[i] + (np.arange(sub) + 0.5) * (edges[i + 1] - edges[i]) / sub
        out[i] = np.mean([sample(L, R, (x - x0) / t, g)[0] for x in xs])
    return out
