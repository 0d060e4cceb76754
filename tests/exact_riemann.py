"""Exact solution of the 1D Riemann problem for an ideal or stiffened gas.

Test infrastructure used to pin the oracle on the Sod shock tube.  Follows
the textbook construction (Toro, "Riemann Solvers and Numerical Methods for
Fluid Dynamics", 3rd ed., 2009, ch. 4): the star pressure is the root of
f_L(p) + f_R(p) + (u_R - u_L) = 0, with f_K the shock (Rankine-Hugoniot)
branch for p > p_K and the rarefaction (isentropic) branch otherwise; the
solution is then sampled on the rays x/t.

The two sides may hold different materials: each has its own gamma and
stiffened-gas constant p_inf (p = (gamma - 1) rho e - gamma p_inf).  The
stiffened gas behaves as an ideal gas in the shifted pressure p + p_inf, so
every wave relation takes p + p_inf in place of p (p_inf = 0: the ideal
gas, the same arithmetic as before).
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, g, pinf=0.0):
    P, Pk = p + pinf, pk + pinf
    c = math.sqrt(g * Pk / rho)
    if p > pk:
        a = 2.0 / ((g + 1.0) * rho)
        b = (g - 1.0) / (g + 1.0) * Pk
        s = math.sqrt(a / (P + b))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (b + P))
    r = P / Pk
    f = 2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * c) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, g, gr=None, pinf_l=0.0, pinf_r=0.0):
    """Star-region pressure and velocity (Newton iteration on p).  g is the
    left gamma and gr the right one (default: g)."""
    gr = g if gr is None else gr
    pmin = 1e-14 - min(pinf_l, pinf_r)
    p = max(1e-12 - min(pinf_l, pinf_r), 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _f_and_df(p, rl, pl, g, pinf_l)
        fr, dfr = _f_and_df(p, rr, pr, gr, pinf_r)
        step = (fl + fr + ur - ul) / (dfl + dfr)
        p_new = max(pmin, p - step)
        if abs(p_new - p) <= 1e-15 * (abs(p_new) + abs(p)):
            p = p_new
            break
        p = p_new
    fl, _ = _f_and_df(p, rl, pl, g, pinf_l)
    fr, _ = _f_and_df(p, rr, pr, gr, pinf_r)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def _side(xi, rk, uk, pk, g, pinf, ps, us, sign):
    """(rho, u, p) on one side of the contact; sign = -1 left, +1 right
    (the right side is the left one mirrored: x -> -x, u -> -u)."""
    gm = (g - 1.0) / (g + 1.0)
    Pk, Ps = pk + pinf, ps + pinf
    c = math.sqrt(g * Pk / rk)
    x, u0, uss = -sign * xi, -sign * uk, -sign * us  # mirrored onto the left
    if ps > pk:  # shock
        s = u0 - c * math.sqrt((g + 1.0) / (2.0 * g) * Ps / Pk + (g - 1.0) / (2.0 * g))
        if x < s:
            return rk, uk, pk
        return rk * (Ps / Pk + gm) / (gm * Ps / Pk + 1.0), us, ps
    cs = c * (Ps / Pk) ** ((g - 1.0) / (2.0 * g))
    if x < u0 - c:
        return rk, uk, pk
    if x > uss - cs:
        return rk * (Ps / Pk) ** (1.0 / g), us, ps
    u = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * u0 + x)
    cc = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * (u0 - x))
    rho = rk * (cc / c) ** (2.0 / (g - 1.0))
    return rho, -sign * u, Pk * (cc / c) ** (2.0 * g / (g - 1.0)) - pinf


def sample(xi, rl, ul, pl, rr, ur, pr, g, gr=None, pinf_l=0.0, pinf_r=0.0):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t for one xi."""
    gr = g if gr is None else gr
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g, gr, pinf_l, pinf_r)
    if xi <= us:  # left of the contact
        return _side(xi, rl, ul, pl, g, pinf_l, ps, us, -1.0)
    return _side(xi, rr, ur, pr, gr, pinf_r, ps, us, 1.0)


def solution(x, t, x0, left, right, g, gr=None, pinf=(0.0, 0.0)):
    """Arrays rho, u, p at positions x and time t > 0."""
    rl, ul, pl = left
    rr, ur, pr = right
    out = np.array([sample((xx - x0) / t, rl, ul, pl, rr, ur, pr, g, gr, *pinf) for xx in np.asarray(x)])
    return out[:, 0], out[:, 1], out[:, 2]


def right_shock_speed(left, right, g, gr=None, pinf=(0.0, 0.0)):
    gr = g if gr is None else gr
    rl, ul, pl = left
    rr, ur, pr = right
    ps, _ = star_state(rl, ul, pl, rr, ur, pr, g, gr, *pinf)
    P, Pr = ps + pinf[1], pr + pinf[1]
    c = math.sqrt(gr * Pr / rr)
    return ur + c * math.sqrt((gr + 1.0) / (2.0 * gr) * P / Pr + (gr - 1.0) / (2.0 * gr))
