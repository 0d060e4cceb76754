"""Self-similar Sedov-Taylor blast wave (spherical, ideal gas, uniform
ambient density, zero ambient pressure), by direct integration.

Test infrastructure: pins the oracle's Sedov runs and, independently, the
energy constant alpha of tests/golden/sedov_alpha.txt.

Construction (Sedov 1959, "Similarity and Dimensional Methods in
Mechanics", ch. IV; written out here from the Euler equations): with
r_s(t) = (E t^2 / (alpha rho0))^(1/5), lambda = r / r_s and x = ln lambda,
seek u = (r/t) v(lambda), rho = rho0 g(lambda), p = rho0 (r/t)^2 P(lambda).
Mass, momentum and the entropy p rho^-gamma carried with the flow give,
with a = v - 2/5 and ' = d/dx,
    a g'/g = -(3 v + v')
    a v'   = v - v^2 - (2 P + P')/g
    P'/P - gamma g'/g = -2 (v - 1)/a,
a linear system for (v', g', P') at each x.  The strong-shock jump at
lambda = 1 (shock speed D = 2 r_s / (5 t)) fixes v = 4/(5(gamma+1)),
g = (gamma+1)/(gamma-1), P = 8/(25(gamma+1)).  Energy conservation gives
alpha = 4 pi int_0^1 (g v^2/2 + P/(gamma-1)) lambda^4 dlambda.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(x, y, gamma):
    v, lg, lp = y  # v, ln g, ln P
    g, p = math.exp(lg), math.exp(lp)
    a = v - 0.4
    q = p / g
    dv = (v - v * v - 2.0 * q + q * (3.0 * gamma * v + 2.0 * (v - 1.0)) / a) / (a - gamma * q / a)
    dlg = -(3.0 * v + dv) / a
    dlp = -(gamma * (3.0 * v + dv) + 2.0 * (v - 1.0)) / a
    return [dv, dlg, dlp]


def profile(gamma=1.4, x_min=-4.0, n=4001):
    """(lambda, v, g, P) from the shock (lambda = 1) inward to e^x_min."""
    y0 = [4.0 / (5.0 * (gamma + 1.0)), math.log((gamma + 1.0) / (gamma - 1.0)),
          math.log(8.0 / (25.0 * (gamma + 1.0)))]
    xs = np.linspace(0.0, x_min, n)
    sol = solve_ivp(_rhs, (0.0, x_min), y0, t_eval=xs, args=(gamma,), rtol=1e-11, atol=1e-13,
                    method="DOP853")
    if not sol.success:
        raise RuntimeError(sol.message)
    lam = np.exp(sol.t)
    return lam, sol.y[0], np.exp(sol.y[1]), np.exp(sol.y[2])


def alpha(gamma=1.4):
    """The energy constant: R(t) = (E / (alpha rho0))^(1/5) t^(2/5)."""
    lam, v, g, p = profile(gamma)
    f = (0.5 * g * v * v + p / (gamma - 1.0)) * lam ** 4
    # lambda decreases along the arrays; below e^-4 the integrand is under 1e-4
    # of its peak and falls like lambda^2, so the tail is under 1e-6 of alpha
    return 4.0 * math.pi * float(np.trapezoid(f[::-1], lam[::-1]))


def density(r, t, energy, gamma=1.4, rho0=1.0):
    """rho(r, t) of the spherical blast of total energy `energy`."""
    lam, _, g, _ = profile(gamma)
    rs = (energy * t * t / (alpha(gamma) * rho0)) ** 0.2
    lr = np.asarray(r, dtype=float) / rs
    out = np.full(lr.shape, rho0)
    inside = lr < 1.0
    out[inside] = rho0 * np.interp(lr[inside], lam[::-1], g[::-1])
    return out


def pressure(r, t, energy, gamma=1.4, rho0=1.0):
    """p(r, t) of the spherical blast (zero ahead of the shock)."""
    lam, _, _, p = profile(gamma)
    rs = (energy * t * t / (alpha(gamma) * rho0)) ** 0.2
    lr = np.asarray(r, dtype=float) / rs
    out = np.zeros(lr.shape)
    inside = lr < 1.0
    out[inside] = rho0 * (rs / t) ** 2 * np.interp(lr[inside], lam[::-1], (p * lam * lam)[::-1])
    return out
