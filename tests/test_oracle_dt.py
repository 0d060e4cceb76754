"""Pins for the oracle's time step (reading R5) and sound speed (reading R2).

The step control takes the CFL limit over the cells,
    dt_cfl = cfl * min_c L_c / sqrt(cs_c^2 + 2 q_c / rho_c),
caps it by growth * dt_last, and caps the first step by dt_init.  The
expected values here come from physics and geometry fixed outside the
oracle's code, not from its formula:

  * An ideal gas at rest has the physical sound speed sqrt(gamma p / rho)
    (gamma (gamma - 1) e with e = p / ((gamma - 1) rho)), no viscosity and,
    on a box cell, L = min(dx, dy, dz) (volume over the largest face).  The
    box below has three different spacings, so a length taken as the
    largest or the middle edge fails.
  * A cell whose energy is negative has no sound speed (max(e, 0)): it
    neither limits the step nor produces a NaN.
  * Under the affine compression u = -alpha (x - x0) every cell, whatever
    its discrete gradient, has div u = tr(-alpha I) = -3 alpha exactly (the
    trilinear volume is cubic in the node positions, so d/dt V(x + t u) =
    V tr(grad u) for an affine u), and a cube has L = h.  The viscosity of
    reading R3 is then q = rho (c_q (3 alpha h)^2 + c_l cs 3 alpha h), and
    the step is cfl h / sqrt(cs^2 + 2 q / rho).  Worked numbers for
    rho = p = 1, gamma = 1.4, h = 1/4, alpha = 2, c_q = 1, c_l = 1/2,
    cfl = 0.3:  cs^2 = 1.4, L div = -1.5, q = 2.25 + 0.75 sqrt(1.4)
    = 3.1374115..., cs^2 + 2 q / rho = 7.6748230..., dt = 0.075 /
    2.7703473... = 0.0270724...  Each coefficient is also switched off on
    its own, so exchanging c_q and c_l, dropping the factor 2 or the q term
    fails.  Expansion (alpha < 0) gives q = 0.
  * The growth cap: with a tiny dt_init on the Sod tube the steps grow by
    exactly the factor 1.1 while the CFL limit (computed here from the
    fields and the node positions) is far away, and no step ever exceeds
    that limit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs


def _box_oracle(md, pd):
    return oracle.Oracle.from_problem(md, pd)


def test_uniform_box_first_dt_is_cfl_min_spacing_over_physical_sound_speed():
    # dx = 0.1, dy = 0.2, dz = 0.05: L must be the smallest spacing
    md = inputs.MeshDesc(6, 5, 4, lo=(0.0, 0.0, 0.0), hi=(0.6, 1.0, 0.2))
    for rho, p, gamma, cfl in ((1.3, 0.7, 1.4, 0.3), (0.2, 5.0, 1.67, 0.45)):
        pd = inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=rho, p_bg=p, gamma=gamma, cfl=cfl)
        o = _box_oracle(md, pd)
        want = cfl * 0.05 / math.sqrt(gamma * p / rho)
        assert abs(o.s.dt - want) <= 1e-14 * want, (o.s.dt, want)
        cs = o.field("cs")
        assert np.max(np.abs(cs - math.sqrt(gamma * p / rho))) <= 1e-14 * math.sqrt(gamma * p / rho)
        # at rest nothing changes, and the growth cap (1.1 dt) does not bind
        rc, n = o.run(max_cycles=3)
        assert rc == 0 and n == 3
        assert abs(o.s.dt - want) <= 1e-14 * want


def test_dt_init_caps_only_the_first_step():
    md = inputs.MeshDesc(4, 4, 4)
    pd = inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, dt_init=1e-3)
    o = _box_oracle(md, pd)
    assert o.s.dt == 1e-3
    rc, _ = o.run(max_cycles=1)
    assert rc == 0
    assert o.s.dt == 1.1 * 1e-3  # grows by exactly the cap


def test_negative_energy_cell_has_no_sound_speed():
    md, pd = inputs.uniform_box(4, rho=1.0, p=1.0)
    o = _box_oracle(md, pd)
    e = o.field("e")
    e[5] = -1e-3
    x, y, z = o.field("x"), o.field("y"), o.field("z")
    zeros = np.zeros_like(x)
    rc = o.set_state(x, y, z, zeros, zeros, zeros, o.field("mn"), o.field("m"), e)
    assert rc == 0
    cs = o.field("cs")
    assert cs[5] == 0.0
    want = 0.3 * 0.25 / math.sqrt(1.4)  # the other cells set the step
    assert abs(o.s.dt - want) <= 1e-14 * want


def _affine_dt(alpha, c_q, c_l, cfl=0.3):
    md = inputs.MeshDesc(4, 4, 4)  # h = 1/4 on the unit cube
    pd = inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=1.0, p_bg=1.0, gamma=1.4, c_q=c_q, c_l=c_l,
                            cfl=cfl)
    o = _box_oracle(md, pd)
    x, y, z = o.field("x"), o.field("y"), o.field("z")
    u, v, w = (-alpha * (c - 0.5) for c in (x, y, z))
    rc = o.set_state(x, y, z, u, v, w, o.field("mn"), o.field("m"), o.field("e"))
    assert rc == 0
    return o


@pytest.mark.parametrize("c_q,c_l,want", [
    # cs^2 + 2 q / rho with cs^2 = 1.4, L |div| = 1.5:
    (1.0, 0.5, 1.4 + 2.0 * (2.25 + 0.75 * math.sqrt(1.4))),   # both terms
    (1.0, 0.0, 1.4 + 2.0 * 2.25),                             # quadratic only
    (0.0, 0.5, 1.4 + 2.0 * 0.75 * math.sqrt(1.4)),            # linear only
])
def test_affine_compression_dt_carries_the_viscosity(c_q, c_l, want):
    o = _affine_dt(2.0, c_q, c_l)
    q = o.field("q")
    q_want = (want - 1.4) / 2.0
    assert np.max(np.abs(q - q_want)) <= 1e-12 * q_want
    dt_want = 0.3 * 0.25 / math.sqrt(want)
    assert abs(o.s.dt - dt_want) <= 1e-13 * dt_want, (o.s.dt, dt_want)
    if c_q == 1.0 and c_l == 0.5:
        assert abs(dt_want - 0.0270724) <= 1e-7  # the worked number of the header


def test_affine_expansion_has_no_viscosity():
    o = _affine_dt(-2.0, 1.0, 0.5)
    assert np.all(o.field("q") == 0.0)
    want = 0.3 * 0.25 / math.sqrt(1.4)
    assert abs(o.s.dt - want) <= 1e-14 * want


def _cfl_limit_from_fields(o, gamma, cfl):
    """cfl * L / sqrt(gamma p / rho + 2 q / rho) per cell, L = min(dx, dy, dz)
    from the node positions (the Sod tube moves along x only, so its cells
    stay boxes)."""
    nx, ny, nz = o.nx, o.ny, o.nz
    x = o.field("x").reshape(nz + 1, ny + 1, nx + 1)
    y = o.field("y").reshape(nz + 1, ny + 1, nx + 1)
    z = o.field("z").reshape(nz + 1, ny + 1, nx + 1)
    dx = np.diff(x, axis=2)[:-1, :-1, :]
    dy = np.diff(y, axis=1)[:-1, :, :-1]
    dz = np.diff(z, axis=0)[:, :-1, :-1]
    L = np.minimum(np.minimum(dx, dy), dz).reshape(-1)
    rho, p, q = o.field("rho"), o.field("p"), o.field("q")
    return float(np.min(cfl * L / np.sqrt(gamma * p / rho + 2.0 * q / rho)))


def test_growth_cap_and_cfl_bound_on_sod():
    md, pd = inputs.sod_x(50, 2, 2)
    pd.dt_init = 1e-6
    o = oracle.Oracle.from_problem(md, pd)
    assert o.s.dt == 1e-6
    grew, bound = 0, 0
    dt_prev = o.s.dt
    for n in range(120):
        rc, done = o.run(max_cycles=1)
        assert rc == 0 and done == 1
        limit = _cfl_limit_from_fields(o, 1.4, 0.3)
        dt = o.s.dt
        assert dt <= limit * (1.0 + 1e-13), (n, dt, limit)
        if 1.1 * dt_prev < limit * (1.0 - 1e-12):
            assert dt == 1.1 * dt_prev, (n, dt, dt_prev)
            grew += 1
        else:
            assert abs(dt - limit) <= 1e-12 * limit, (n, dt, limit)
            bound += 1
        dt_prev = dt
    # both regimes were exercised
    assert grew >= 50 and bound >= 10, (grew, bound)
