"""Oracle pins for several materials (reading R18: per-material stiffened
gas EoS, mixed cells closed by uniform strain, donor-cell remap of each
material's volume, mass and energy, a 1e-8 fraction cutoff).

What fixes each expected value:
  * the exact Riemann solution with a different gamma and stiffened-gas
    constant on each side; the solver itself is checked against the
    Rankine-Hugoniot conditions across its shock, the isentropic
    invariants across its fan and the mirror symmetry x -> -x;
  * splitting one gas into two identical materials, in any fractions,
    changes nothing: the single-material oracle;
  * mixed cells in pressure equilibrium stay at rest;
  * a uniform translation of the mesh remaps each volume fraction as the
    textbook 1D first-order upwind scheme does and keeps every material's
    density and energy;
  * uniform compression of a uniformly mixed column: every material
    follows its own adiabat (p + p_inf) V_k^gamma = const, the error
    falling at first order in dt;
  * the first dt of a box at rest, CFL h / c: the stiffened gas's
    c^2 = gamma (p + p_inf) / rho and the mass-weighted mixture c^2;
  * conservation of the total mass and energy, and of each material's
    mass up to the fragments the cutoff moves.
"""
import dataclasses
import math

import numpy as np
import pytest

import exact_riemann as er
import oracle
from paper_2209_01983_gb300 import inputs

# Sod states with a stiffened gas on one side (A: the high-pressure left,
# B: the low-pressure right; B's end time keeps its fast shock off the wall)
LEFT, RIGHT = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
CASES = {"A": ((3.0, 1.4), (0.5, 0.0), 0.2), "B": ((1.4, 3.0), (0.0, 0.3), 0.1)}


def mat_problem(pd, gam, pinf):
    return dataclasses.replace(pd, nmat=2, mat_gamma=(gam[0], gam[1], 1.4, 1.4),
                               mat_pinf=(pinf[0], pinf[1], 0.0, 0.0))


def stiff_e(p, rho, g, pinf):
    """Specific energy of the stiffened gas at (rho, p), its EoS solved."""
    return (p + g * pinf) / ((g - 1.0) * rho)


def stiff_p(rho, e, g, pinf):
    return (g - 1.0) * rho * e - g * pinf


# ---------------------------------------------------------------------------
# The exact solver with two materials
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_solver_jump_conditions_and_fan(case):
    (gl, gr), (pl_inf, pr_inf), _ = CASES[case]
    args = (*LEFT, *RIGHT, gl, gr, pl_inf, pr_inf)
    ps, us = er.star_state(*args)
    assert ps > RIGHT[2] and ps < LEFT[2]  # right shock, left fan
    # Rankine-Hugoniot across the right shock, in the shock's frame
    S = er.right_shock_speed(LEFT, RIGHT, gl, gr, (pl_inf, pr_inf))
    r1, u1, p1 = er.sample(S + 1e-9, *args)
    r2, u2, p2 = er.sample(S - 1e-9, *args)
    assert (r1, u1, p1) == RIGHT and p2 == ps and u2 == us
    w1, w2 = u1 - S, u2 - S
    assert r1 * w1 == pytest.approx(r2 * w2, rel=1e-12)
    assert p1 + r1 * w1 * w1 == pytest.approx(p2 + r2 * w2 * w2, rel=1e-12)
    h1 = stiff_e(p1, r1, gr, pr_inf) + p1 / r1
    h2 = stiff_e(p2, r2, gr, pr_inf) + p2 / r2
    assert h1 + 0.5 * w1 * w1 == pytest.approx(h2 + 0.5 * w2 * w2, rel=1e-12)
    # across the left fan: (p + p_inf) / rho^gamma and u + 2 c / (gamma - 1)
    cl = math.sqrt(gl * (LEFT[2] + pl_inf) / LEFT[0])
    rs = er.sample(us - 1e-9, *args)[0]
    cstar = math.sqrt(gl * (ps + pl_inf) / rs)
    ent, inv = [], []
    for xi in np.linspace(-cl, us - cstar, 7):
        r, u, p = er.sample(xi, *args)
        ent.append((p + pl_inf) / r ** gl)
        inv.append(u + 2.0 * math.sqrt(gl * (p + pl_inf) / r) / (gl - 1.0))
    assert np.ptp(ent) <= 1e-12 * ent[0]
    assert np.ptp(inv) <= 1e-12 * inv[0]


def test_exact_solver_mirror_symmetry():
    (gl, gr), (pl_inf, pr_inf), _ = CASES["A"]
    # the same problem mirrored: high pressure on the right
    for xi in np.linspace(-3.0, 3.0, 41):
        a = er.sample(xi, *LEFT, *RIGHT, gl, gr, pl_inf, pr_inf)
        b = er.sample(-xi, *RIGHT, *LEFT, gr, gl, pr_inf, pl_inf)
        assert b[0] == pytest.approx(a[0], rel=1e-12)
        assert b[1] == pytest.approx(-a[1], rel=1e-12, abs=1e-14)
        assert b[2] == pytest.approx(a[2], rel=1e-12)


# ---------------------------------------------------------------------------
# Two-material shock tubes against the exact solution
# ---------------------------------------------------------------------------

def sod2(case, nx, remap_every):
    gam, pinf, t_end = CASES[case]
    md, pd = inputs.sod_x(nx, 4, 4)
    o = oracle.Oracle.from_problem(md, mat_problem(pd, gam, pinf))
    d0 = o.diagnostics()
    mats0 = [o.field("m0").sum(), o.field("m1").sum()]
    rc, _ = o.run(t_end=t_end, max_cycles=3000, remap_every=remap_every)  # these runs take at most ~320
    assert rc == 0 and o.s.t == t_end
    x = o.field("x").reshape(5, 5, nx + 1)[0, 0]
    xc = 0.5 * (x[:-1] + x[1:])  # the tube moves along x only
    rho = o.field("rho").reshape(4, 4, nx)[0, 0]
    rex, _, _ = er.solution(xc, t_end, 0.5, LEFT, RIGHT, gam[0], gam[1], pinf)
    l1 = float(np.sum(np.abs(rho - rex) * np.diff(x)))
    return o, d0, mats0, l1, x


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_material_sod_lagrange(case):
    gam, pinf, t_end = CASES[case]
    errs = []
    for nx in (50, 100, 200):
        o, d0, mats0, l1, x = sod2(case, nx, 0)
        errs.append(l1)
        # cells stay pure; the interface node moves with the contact
        a1 = o.field("alpha1").reshape(4, 4, nx)[0, 0]
        assert set(np.unique(a1)) == {0.0, 1.0}
        i_if = int(np.argmax(a1 > 0.5))
        _, us = er.star_state(*LEFT, *RIGHT, gam[0], gam[1], *pinf)
        assert abs(x[i_if] - (0.5 + us * t_end)) <= 0.5 / nx
        d = o.diagnostics()
        assert d["mass"] == d0["mass"]
        assert abs(d["etot"] - d0["etot"]) <= 1e-13 * d0["etot"]
        assert [o.field("m0").sum(), o.field("m1").sum()] == mats0
    assert errs[1] <= 8e-3
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.75 * errs[0] / 1.5


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_material_sod_eulerian(case):
    gam, pinf, t_end = CASES[case]
    errs = []
    for nx in (50, 100, 200):
        o, d0, mats0, l1, x = sod2(case, nx, 1)
        errs.append(l1)
        a0, a1 = o.field("alpha0"), o.field("alpha1")
        assert np.all((a0 >= 0.0) & (a0 <= 1.0) & (a1 >= 0.0) & (a1 <= 1.0))
        assert np.max(np.abs(a0 + a1 - 1.0)) <= 1e-15
        assert np.sum((a1 > 0.0) & (a1 < 1.0)) > 0  # the contact smears into mixed cells
        # the material-1 volume against the exact contact position
        _, us = er.star_state(*LEFT, *RIGHT, gam[0], gam[1], *pinf)
        v1 = float(np.sum(a1 * o.field("vol")))
        area = 0.04 * 0.04
        assert abs(v1 / area - (1.0 - (0.5 + us * t_end))) <= 1.5 / nx
        d = o.diagnostics()
        assert d["mass"] == pytest.approx(d0["mass"], rel=1e-14)
        assert abs(d["etot"] - d0["etot"]) <= 1e-13 * d0["etot"]
        for m_now, m_start in zip([o.field("m0").sum(), o.field("m1").sum()], mats0):
            assert m_now == pytest.approx(m_start, rel=1e-7)  # up to fragments under the cutoff
    assert errs[1] <= 2e-2
    assert errs[0] > errs[1] > errs[2]


# ---------------------------------------------------------------------------
# Invariances
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("remap_every,c_hg,time_order", [(1, 0.0, 1), (3, 0.0, 1), (1, 0.05, 1), (1, 0.0, 2),
                                                         (3, 0.05, 2)])
def test_identical_materials_equal_one_gas(remap_every, c_hg, time_order):
    md, pd = inputs.sedov_octant(1, jitter=0.1)
    md.nx, md.ny, md.nz = 14, 12, 10
    pd = dataclasses.replace(pd, c_hg=c_hg, time_order=time_order)
    one = oracle.Oracle.from_problem(md, pd)
    two = oracle.Oracle.from_problem(md, mat_problem(pd, (1.4, 1.4), (0.0, 0.0)))
    # random fractions and mass shares with one specific energy per cell
    rng = np.random.default_rng(2209)
    a0, f0 = rng.random(md.ncell), rng.random(md.ncell)
    m, e = two.field("m"), two.field("e")
    assert two.set_materials([a0, 1.0 - a0], [f0 * m, (1.0 - f0) * m], [e, e]) == 0
    for o in (one, two):
        rc, n = o.run(max_cycles=40, remap_every=remap_every)
        assert rc == 0 and n == 40
    for f in ("x", "u", "v", "w", "mn", "m", "e", "rho", "p", "q", "cs", "vol"):
        a, b = two.field(f), one.field(f)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), f
    assert two.s.dt == pytest.approx(one.s.dt, rel=1e-12)


def mixed_box(nx, ny, nz, jitter, gam, pinf, rho, p, reflect=(1, 1, 1, 1, 1, 1), c_q=1.0, c_l=0.5, frac=None,
              hi=(1.0, 1.0, 1.0), time_order=1):
    """Box at rest whose cells hold both materials at pressure p, material
    k at density rho[k], fractions frac (default: random in [0.1, 0.9])."""
    md = inputs.MeshDesc(nx, ny, nz, lo=(0.0, 0.0, 0.0), hi=hi, jitter=jitter, reflect=reflect)
    pd = mat_problem(inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=rho[0], p_bg=p, c_q=c_q, c_l=c_l,
                                        time_order=time_order), gam, pinf)
    o = oracle.Oracle.from_problem(md, pd)
    rng = np.random.default_rng(7)
    a0 = rng.uniform(0.1, 0.9, md.ncell) if frac is None else np.full(md.ncell, frac)
    vol = o.field("vol")
    alpha = [a0, 1.0 - a0]
    mm = [alpha[k] * rho[k] * vol for k in range(2)]
    me = [np.full(md.ncell, stiff_e(p, rho[k], gam[k], pinf[k])) for k in range(2)]
    assert o.set_materials(alpha, mm, me) == 0
    # node masses of the new cell masses, an eighth of each cell's
    nxn, nyn = nx + 1, ny + 1
    mc = o.field("m").reshape(nz, ny, nx) / 8.0
    mn = np.zeros((nz + 1, ny + 1, nx + 1))
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                mn[dk:dk + nz, dj:dj + ny, di:di + nx] += mc
    assert (nxn, nyn) == (nx + 1, ny + 1)
    zero = np.zeros(md.nnode)
    assert o.set_state(o.field("x"), o.field("y"), o.field("z"), zero, zero, zero, mn.reshape(-1), o.field("m"),
                       o.field("e")) == 0
    return md, o


@pytest.mark.parametrize("remap_every", [0, 1])
def test_pressure_equilibrium_stays_at_rest(remap_every):
    md, o = mixed_box(9, 8, 7, 0.1, (1.4, 3.0), (0.0, 0.5), (1.0, 3.0), 1.0)
    rc, n = o.run(max_cycles=20, remap_every=remap_every)
    assert rc == 0 and n == 20
    c = math.sqrt(3.0 * 1.5 / 3.0)
    for f in ("u", "v", "w"):
        assert np.max(np.abs(o.field(f))) <= 1e-13 * c, f
    assert np.max(np.abs(o.field("p") - 1.0)) <= 1e-13
    assert np.max(np.abs(o.field("q"))) <= 1e-14  # viscosity of roundoff-sized motion


def test_translation_remap_is_upwind_advection():
    nx, nu, steps = 40, 0.3, 10
    gam, pinf, rho, p = (1.4, 3.0), (0.0, 0.5), (1.0, 2.5), 1.0
    md, o = mixed_box(nx, 3, 3, 0.0, gam, pinf, rho, p, frac=1.0, hi=(1.0, 0.075, 0.075))
    # pure cells: material 1 from x = 0.5
    vol = o.field("vol")
    right = (np.arange(md.ncell) % nx) >= nx // 2
    a1 = right.astype(float)
    mm = [(1.0 - a1) * rho[0] * vol, a1 * rho[1] * vol]
    me = [np.where(right, 0.0, stiff_e(p, rho[0], gam[0], pinf[0])),
          np.where(right, stiff_e(p, rho[1], gam[1], pinf[1]), 0.0)]
    assert o.set_materials([1.0 - a1, a1], mm, me) == 0
    h = 1.0 / nx
    ref = a1.reshape(3, 3, nx)[0, 0].copy()
    zero = np.zeros(md.nnode)
    for _ in range(steps):
        # the mesh shifted by nu h along x, at rest, then remapped back
        assert o.set_state(o.field("xr") + nu * h, o.field("yr"), o.field("zr"), zero, zero, zero, o.field("mn"),
                           o.field("m"), o.field("e")) == 0
        assert o.remap_step() == 0
        new = ref.copy()
        new[1:nx - 1] = (1.0 - nu) * ref[1:nx - 1] + nu * ref[0:nx - 2]
        ref = new
    got = o.field("alpha1").reshape(3, 3, nx)
    inner = slice(1, nx - 1)
    assert np.max(np.abs(got[:, :, inner] - ref[inner])) <= 1e-13
    assert np.sum((ref > 0.0) & (ref < 1.0)) >= steps  # the front has spread
    # every material keeps its density and specific energy where present,
    # beyond the cells fed from the wall cell (which only loses, so thins)
    vol = o.field("vol")
    far = slice(steps + 1, nx - 1)
    for k in range(2):
        a, m_k, e_k = (o.field(f"{q}{k}").reshape(3, 3, nx)[:, :, far] for q in ("alpha", "m", "e"))
        v = vol.reshape(3, 3, nx)[:, :, far]
        there = a > 0.0
        assert np.max(np.abs(m_k[there] / (a[there] * v[there]) / rho[k] - 1.0)) <= 1e-12
        e_ref = stiff_e(p, rho[k], gam[k], pinf[k])
        assert np.max(np.abs(e_k[there] / e_ref - 1.0)) <= 1e-12


def test_uniform_compression_follows_each_adiabat():
    """A column of uniformly mixed cells compressed at a constant rate
    u = -beta x (x-lo a symmetry plane, x-hi free, no viscosity): away from
    the free end the motion stays affine, every cell keeps its fractions
    and each material follows its own adiabat.  The single-stage step is
    first order in time, so halving dt halves the error."""
    nx, beta, t_end = 120, 2.0, 0.1  # V / V0 = 0.8 at the end
    gam, pinf, rho, p0 = (1.4, 3.0), (0.0, 0.5), (1.0, 2.0), 1.0
    errs = []
    for steps in (40, 80):
        md, o = mixed_box(nx, 1, 1, 0.0, gam, pinf, rho, p0, reflect=(1, 0, 1, 1, 1, 1), c_q=0.0, c_l=0.0,
                          frac=0.4, hi=(1.0, 1.0 / nx, 1.0 / nx))
        v0 = o.field("vol")[0]
        x = o.field("x")
        zero = np.zeros(md.nnode)
        assert o.set_state(x, o.field("y"), o.field("z"), -beta * x, zero, zero, o.field("mn"), o.field("m"),
                           o.field("e")) == 0
        for _ in range(steps):
            assert o.lagrange_step(t_end / steps) == 0
        inner = np.arange(nx - steps - 3)  # cells the free end has not reached
        vol = o.field("vol")[inner]
        assert np.max(np.abs(vol / (v0 * (1.0 - beta * t_end)) - 1.0)) <= 1e-9  # roundoff growth
        err = 0.0
        for k, a in enumerate((0.4, 0.6)):
            assert np.all(o.field(f"alpha{k}")[inner] == a)
            rho_k = o.field(f"m{k}")[inner] / (a * vol)
            p_k = stiff_p(rho_k, o.field(f"e{k}")[inner], gam[k], pinf[k])
            p_adiabat = (p0 + pinf[k]) * (v0 / vol) ** gam[k] - pinf[k]
            err = max(err, float(np.max(np.abs(p_k / p_adiabat - 1.0))))
        errs.append(err)
    assert errs[0] <= 5e-3
    assert 0.4 * errs[0] <= errs[1] <= 0.6 * errs[0]


def test_predictor_corrector_is_second_order_for_each_material():
    """The uniformly compressed mixed column of the adiabat test with the
    predictor-corrector: each material still follows its own adiabat, now
    with an error falling at second order in dt (the half-step pressures of
    every material enter the corrector's work split)."""
    nx, beta, t_end = 120, 2.0, 0.1
    gam, pinf, rho, p0 = (1.4, 3.0), (0.0, 0.5), (1.0, 2.0), 1.0
    errs = []
    for steps in (20, 40):
        md, o = mixed_box(nx, 1, 1, 0.0, gam, pinf, rho, p0, reflect=(1, 0, 1, 1, 1, 1), c_q=0.0, c_l=0.0,
                          frac=0.4, hi=(1.0, 1.0 / nx, 1.0 / nx), time_order=2)
        v0 = o.field("vol")[0]
        x = o.field("x")
        zero = np.zeros(md.nnode)
        assert o.set_state(x, o.field("y"), o.field("z"), -beta * x, zero, zero, o.field("mn"), o.field("m"),
                           o.field("e")) == 0
        for _ in range(steps):
            assert o.lagrange_step(t_end / steps) == 0
        inner = np.arange(nx - 2 * steps - 3)  # the corrector reaches two cells a step
        vol = o.field("vol")[inner]
        err = 0.0
        for k, a in enumerate((0.4, 0.6)):
            rho_k = o.field(f"m{k}")[inner] / (a * vol)
            p_k = stiff_p(rho_k, o.field(f"e{k}")[inner], gam[k], pinf[k])
            p_adiabat = (p0 + pinf[k]) * (v0 / vol) ** gam[k] - pinf[k]
            err = max(err, float(np.max(np.abs(p_k / p_adiabat - 1.0))))
        errs.append(err)
    assert errs[0] <= 5e-4
    assert errs[1] <= 0.35 * errs[0]  # second order: a quarter


def test_mixed_column_standing_wave_period():
    """A small standing wave u = eps sin(pi x) in a column of uniformly
    mixed cells between walls (no viscosity) oscillates at the uniform-strain
    mixture's sound speed, c^2 = sum_k m_k c_k^2 / m = sum_k alpha_k rho_k
    c_k^2 / rho, so the kinetic energy first vanishes at t = L / (2 c).
    Worked numbers: alpha = (0.4, 0.6), rho = (1, 2), p = 1, gamma = (1.4, 3),
    p_inf = (0, 2): c_0^2 = 1.4, c_1^2 = 3 (1 + 2) / 2 = 4.5, c^2 = (0.4 1.4 +
    1.2 4.5) / 1.6 = 3.725, t = 0.5 / 1.93003 = 0.25906.  A volume-weighted
    c^2 (3.26, t = 0.2769) or Wood's pressure-equilibrium speed (c^2 = 1.774,
    t = 0.3754) each miss by more than 6%."""
    nx = 100
    gam, pinf, rho, p = (1.4, 3.0), (0.0, 2.0), (1.0, 2.0), 1.0
    md, o = mixed_box(nx, 1, 1, 0.0, gam, pinf, rho, p, c_q=0.0, c_l=0.0, frac=0.4, hi=(1.0, 1.0 / nx, 1.0 / nx))
    x = o.field("x")
    zero = np.zeros(md.nnode)
    assert o.set_state(x, o.field("y"), o.field("z"), 1e-4 * np.sin(math.pi * x), zero, zero, o.field("mn"),
                       o.field("m"), o.field("e")) == 0
    ts, ks = [o.s.t], [o.diagnostics()["ke"]]
    while o.s.t < 0.33:
        rc, n = o.run(max_cycles=1)
        assert rc == 0 and n == 1
        ts.append(o.s.t)
        ks.append(o.diagnostics()["ke"])
    ks = np.array(ks)
    i = int(np.argmin(ks))
    assert 0 < i < len(ks) - 1
    t0, t1, t2 = ts[i - 1], ts[i], ts[i + 1]  # the parabola through the samples around the minimum
    k0, k1, k2 = ks[i - 1], ks[i], ks[i + 1]
    den = (t0 - t1) * (t0 - t2) * (t1 - t2)
    A = (t2 * (k1 - k0) + t1 * (k0 - k2) + t0 * (k2 - k1)) / den
    B = (t2 * t2 * (k0 - k1) + t1 * t1 * (k2 - k0) + t0 * t0 * (k1 - k2)) / den
    t_min = -B / (2.0 * A)
    c2 = (0.4 * 1.0 * 1.4 + 0.6 * 2.0 * 4.5) / (0.4 * 1.0 + 0.6 * 2.0)
    want = 0.5 / math.sqrt(c2)
    assert abs(want - 0.25906) <= 1e-5
    assert abs(t_min - want) <= 0.01 * want, (t_min, want)
    assert ks[i] <= 1e-3 * ks[0]


def test_first_dt_closed_forms():
    # unequal spacings: h = min(1/8, 0.6/6, 0.4/5) = 0.08
    hi = (1.0, 0.6, 0.4)
    gam, pinf = (1.4, 3.0), (0.0, 2.0)
    md = inputs.MeshDesc(8, 6, 5, lo=(0.0, 0.0, 0.0), hi=hi)
    pd = mat_problem(inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=1.0, p_bg=1.0, x_split=0.5), gam, pinf)
    o = oracle.Oracle.from_problem(md, pd)
    # pure cells: the stiffened gas's c^2 = gamma (p + p_inf) / rho = 9 bounds dt
    assert o.cfl_dt() == pytest.approx(0.3 * 0.08 / 3.0, rel=1e-13)
    e1 = o.field("e1")[o.field("alpha1") > 0.0]
    assert np.all(e1 == stiff_e(1.0, 1.0, 3.0, 2.0))
    # uniformly mixed: c^2 = sum_k m_k c_k^2 / m
    _, o = mixed_box(8, 6, 5, 0.0, gam, pinf, (1.0, 2.0), 1.0, frac=0.3, hi=hi)
    c2 = (0.3 * 1.0 * 1.4 + 0.7 * 2.0 * (3.0 * 3.0 / 2.0)) / (0.3 * 1.0 + 0.7 * 2.0)
    assert o.cfl_dt() == pytest.approx(0.3 * 0.08 / math.sqrt(c2), rel=1e-13)
    assert np.max(np.abs(o.field("p") - 1.0)) <= 1e-14


def test_two_material_sedov_conservation():
    md, pd = inputs.sedov_octant(16, jitter=0.1)
    pd = dataclasses.replace(mat_problem(pd, (1.4, 1.67), (0.0, 0.0)), x_split=0.3)
    o = oracle.Oracle.from_problem(md, pd)
    d0 = o.diagnostics()
    mats0 = [o.field("m0").sum(), o.field("m1").sum()]
    rc, n = o.run(max_cycles=80, remap_every=1)
    assert rc == 0 and n == 80
    d = o.diagnostics()
    assert d["mass"] == pytest.approx(d0["mass"], rel=1e-14)
    assert abs(d["etot"] - d0["etot"]) <= 1e-12 * d0["etot"]
    for m_now, m_start in zip([o.field("m0").sum(), o.field("m1").sum()], mats0):
        assert m_now == pytest.approx(m_start, rel=1e-7)
    a0, a1 = o.field("alpha0"), o.field("alpha1")
    assert np.all((a1 == 0.0) | (a1 > 1e-8)) and np.all((a0 == 0.0) | (a0 > 1e-8))
    assert np.max(np.abs(a0 + a1 - 1.0)) <= 1e-15
    assert np.sum((a1 > 0.0) & (a1 < 1.0)) > 0
    # cell totals are the materials' sums
    m_sum = o.field("m0") + o.field("m1")
    assert np.max(np.abs(m_sum - o.field("m"))) <= 1e-15 * np.max(o.field("m"))
    ie = o.field("m0") * o.field("e0") + o.field("m1") * o.field("e1")
    assert np.max(np.abs(ie - o.field("m") * o.field("e"))) <= 1e-14 * np.max(np.abs(ie))


@pytest.mark.parametrize("remap_every,time_order", [(0, 1), (1, 1), (0, 2), (1, 2)])
def test_energy_exact_with_hourglass_control(remap_every, time_order):
    # hourglass control on a jittered two-material blast: the materials share
    # the hourglass forces' work by fraction, the cell total stays the
    # compatible one, so the total energy is exact; with the
    # predictor-corrector the shares are those of the half step
    md, pd = inputs.sedov_octant(16, jitter=0.1)
    pd = dataclasses.replace(mat_problem(pd, (1.4, 3.0), (0.0, 1e-6)), x_split=0.2, c_hg=0.1, time_order=time_order)
    o = oracle.Oracle.from_problem(md, pd)
    d0 = o.diagnostics()
    rc, n = o.run(max_cycles=60, remap_every=remap_every)
    assert rc == 0 and n == 60
    d = o.diagnostics()
    assert abs(d["etot"] - d0["etot"]) <= 1e-12 * d0["etot"]
    assert d["mass"] == pytest.approx(d0["mass"], rel=1e-14)


def test_rules():
    md, pd = inputs.sod_x(10, 2, 2)
    base = mat_problem(pd, (1.4, 3.0), (0.0, 0.5))
    for bad in (dict(remap_order=2), dict(shear0=1.0),
                dict(mat_gamma=(1.0, 3.0, 1.4, 1.4)), dict(mat_pinf=(-1.0, 0.0, 0.0, 0.0))):
        with pytest.raises(RuntimeError):
            oracle.Oracle.from_problem(md, dataclasses.replace(base, **bad))
    o = oracle.Oracle.from_problem(md, base)
    nc = md.ncell
    ones, zeros = np.ones(nc), np.zeros(nc)
    m, e = o.field("m"), o.field("e")
    assert o.set_materials([ones, zeros], [m, zeros], [e, zeros]) == 0
    assert o.set_materials([ones, ones], [m, m], [e, e]) == oracle.EINVAL  # fractions sum to 2
    assert o.set_materials([ones, zeros], [m, m], [e, e]) == oracle.EINVAL  # mass without volume
    # a single-material problem has no material fields
    o1 = oracle.Oracle.from_problem(md, pd)
    with pytest.raises(KeyError):
        o1.field("alpha0")
