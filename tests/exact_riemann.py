"""Exact solution of the 1D Riemann problem for an ideal gas.

Test infrastructure used to pin the oracle on the Sod shock tube.  Follows
the textbook construction (Toro, "Riemann Solvers and Numerical Methods for
Fluid Dynamics", 3rd ed., 2009, ch. 4): the star pressure is the root of
f_L(p) + f_R(p) + (u_R - u_L) = 0, with f_K the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic) branch otherwise; the
solution is then sampled on the rays x/t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, g):
    c = math.sqrt(g * pk / rho)
    if p > pk:
        a = 2.0 / ((g + 1.0) * rho)
        b = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(a / (p + b))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (b + p))
    r = p / pk
    f = 2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * c) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, g):
    """Star-region pressure and velocity (Newton iteration on p)."""
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _f_and_df(p, rl, pl, g)
        fr, dfr = _f_and_df(p, rr, pr, g)
        step = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(1e-14, p - step)
        if abs(p_new - p) <= 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f_and_df(p, rl, pl, g)
    fr, _ = _f_and_df(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, rl, ul, pl, rr, ur, pr, g):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t for one xi."""
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g)
    gm = (g - 1.0) / (g + 1.0)
    if xi <= us:  # left of the contact
        c = math.sqrt(g * pl / rl)
        if ps > pl:  # left shock
            sl = ul - c * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            if xi < sl:
                return rl, ul, pl
            return rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
        cs = c * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        if xi < ul - c:
            return rl, ul, pl
        if xi > us - cs:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        u = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * ul + xi)
        cc = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * (ul - xi))
        rho = rl * (cc / c) ** (2.0 / (g - 1.0))
        return rho, u, pl * (cc / c) ** (2.0 * g / (g - 1.0))
    c = math.sqrt(g * pr / rr)
    if ps > pr:  # right shock
        sr = ur + c * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        if xi > sr:
            return rr, ur, pr
        return rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
    cs = c * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    if xi > ur + c:
        return rr, ur, pr
    if xi < us + cs:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    u = 2.0 / (g + 1.0) * (-c + 0.5 * (g - 1.0) * ur + xi)
    cc = 2.0 / (g + 1.0) * (c - 0.5 * (g - 1.0) * (ur - xi))
    rho = rr * (cc / c) ** (2.0 / (g - 1.0))
    return rho, u, pr * (cc / c) ** (2.0 * g / (g - 1.0))


def solution(x, t, x0, left, right, g):
    """Arrays rho, u, p at positions x and time t > 0."""
    rl, ul, pl = left
    rr, ur, pr = right
    out = np.array([sample((xx - x0) / t, rl, ul, pl, rr, ur, pr, g) for xx in np.asarray(x)])
    return out[:, 0], out[:, 1], out[:, 2]


def right_shock_speed(left, right, g):
    rl, ul, pl = left
    rr, ur, pr = right
    ps, _ = star_state(rl, ul, pl, rr, ur, pr, g)
    c = math.sqrt(g * pr / rr)
    return ur + c * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
