"""Several materials on the GPU (FP64 general kernels) against the oracle,
element by element, through the C ABI.

Per-material fields are compared as volume fraction alpha_k, mass m_k and
internal energy m_k e_k, each relative to its own maximum (1e-10, as every
other FP64 field).  The specific energy e_k of a fragment near the 1e-8
fraction cutoff is the ratio of two small numbers and carries the rounding
of the fluxes that made it, so it is compared through m_k e_k.  The oracle
side of each case is pinned in test_oracle_multimat.py.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs
from test_gpu_parity import CELL_FIELDS, NODE_FIELDS, compare

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def mat_problem(pd, gam, pinf, **extra):
    return dataclasses.replace(pd, nmat=len(gam), mat_gamma=tuple(gam) + (1.4,) * (4 - len(gam)),
                               mat_pinf=tuple(pinf) + (0.0,) * (4 - len(pinf)), **extra)


def compare_materials(st, o, nmat, tol=TOL):
    errs = {}
    for k in range(nmat):
        a_g, a_o = st.field(f"alpha{k}"), o.field(f"alpha{k}")
        m_g, m_o = st.field(f"m{k}"), o.field(f"m{k}")
        ie_g, ie_o = m_g * st.field(f"e{k}"), m_o * o.field(f"e{k}")
        for name, g, r in ((f"alpha{k}", a_g, a_o), (f"m{k}", m_g, m_o), (f"ie{k}", ie_g, ie_o)):
            scale = float(np.max(np.abs(r)))
            errs[name] = float(np.max(np.abs(g - r))) / scale if scale > 0 else float(np.max(np.abs(g)))
        # presence decided alike on both sides
        assert np.array_equal(a_g > 0.0, a_o > 0.0), k
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"material fields over {tol}: {bad}"
    return errs


def run_both(sale, md, pd, cycles=None, t_end=None, remap_every=0):
    st = sale.State(md, pd)
    o = oracle.Oracle.from_problem(md, pd)
    kw = dict(remap_every=remap_every)
    if cycles is not None:
        kw["max_cycles"] = cycles
    if t_end is not None:
        kw["t_end"] = t_end
    n = st.run_to_time(**kw)
    rc, n_o = o.run(**kw)
    assert rc == 0 and n == n_o
    return st, o


@pytest.mark.parametrize("remap_every", [0, 1])
def test_two_material_sod_against_oracle(sale, remap_every):
    # stiffened gas on the high-pressure side, ideal gas on the other
    md, pd = inputs.sod_x(100, 4, 4)
    pd = mat_problem(pd, (3.0, 1.4), (0.5, 0.0))
    st, o = run_both(sale, md, pd, t_end=0.2, remap_every=remap_every)
    assert st.diagnostics()["t"] == 0.2
    compare(st, o)
    compare_materials(st, o, 2)
    if remap_every:
        a1 = st.field("alpha1")
        assert np.sum((a1 > 0.0) & (a1 < 1.0)) > 0


@pytest.mark.parametrize("remap_every,cycles", [(1, 60), (3, 60), (0, 40)])
def test_two_material_sedov_against_oracle(sale, remap_every, cycles):
    md = inputs.MeshDesc(16, 13, 11, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    pd = mat_problem(pd, (1.4, 1.67), (0.0, 0.0), x_split=0.3)
    st, o = run_both(sale, md, pd, cycles=cycles, remap_every=remap_every)
    compare(st, o)
    compare_materials(st, o, 2)
    assert st.diagnostics()["dt"] == pytest.approx(o.s.dt, rel=1e-10)


@pytest.mark.parametrize("remap_every,cycles", [(1, 40), (3, 45), (0, 40)])
def test_two_materials_with_hourglass_control(sale, remap_every, cycles):
    """Hourglass control with two materials (the hourglass work shared by
    fraction, the mixture's sound speed in its coefficient)."""
    md = inputs.MeshDesc(15, 13, 11, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    pd = mat_problem(pd, (1.4, 3.0), (0.0, 1e-6), x_split=0.2, c_hg=0.1)
    st, o = run_both(sale, md, pd, cycles=cycles, remap_every=remap_every)
    compare(st, o)
    compare_materials(st, o, 2)
    d0, d1 = sale.State(md, pd).diagnostics(), st.diagnostics()
    assert abs(d1["etot"] - d0["etot"]) <= 1e-12 * abs(d0["etot"])


@pytest.mark.parametrize("remap_every,cycles,c_hg", [(1, 40, 0.0), (3, 45, 0.0), (0, 40, 0.0), (1, 30, 0.1)])
def test_two_materials_with_predictor_corrector(sale, remap_every, cycles, c_hg):
    """The predictor-corrector step with two materials: each material's
    half-step energy and share of sigma from the predictor enter the
    corrector's work split."""
    md = inputs.MeshDesc(15, 13, 11, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    pd = mat_problem(pd, (1.4, 3.0), (0.0, 1e-6), x_split=0.2, time_order=2, c_hg=c_hg)
    st, o = run_both(sale, md, pd, cycles=cycles, remap_every=remap_every)
    compare(st, o)
    compare_materials(st, o, 2)
    d0, d1 = sale.State(md, pd).diagnostics(), st.diagnostics()
    assert abs(d1["etot"] - d0["etot"]) <= 1e-12 * abs(d0["etot"])


def test_explicit_steps_then_eulerian_cycles(sale):
    """Explicit Lagrangian steps with given dt and remaps (general kernels),
    then Eulerian cycles from the reference mesh (cached-geometry kernels):
    the two kernel sets hand the material state to each other."""
    md = inputs.MeshDesc(14, 12, 10, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    pd = mat_problem(pd, (1.4, 3.0), (0.0, 1e-5), x_split=0.2)
    st = sale.State(md, pd)
    o = oracle.Oracle.from_problem(md, pd)
    for it in range(6):
        dt = 2e-4 * (1 + it)
        st.lagrange_step(dt)
        o.check(o.lagrange_step(dt))
        if it % 2 == 1:
            st.remap_step()
            o.check(o.remap_step())
    compare(st, o)
    compare_materials(st, o, 2)
    assert st.run_to_time(max_cycles=20, remap_every=1) == 20
    rc, n = o.run(max_cycles=20, remap_every=1)
    assert rc == 0 and n == 20
    compare(st, o)
    compare_materials(st, o, 2)


@pytest.mark.parametrize("nmat", [3, 4])
def test_materials_from_uploaded_fractions(sale, nmat):
    """Fractions, masses and energies uploaded through sale_set_field (a
    random mixture of three or four materials, some stiffened, at one
    pressure) drive the following Eulerian cycles exactly as the oracle's
    set_materials does."""
    md = inputs.MeshDesc(14, 12, 10, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    gam, pinf, rho = (1.4, 3.0, 2.2, 5.0 / 3.0)[:nmat], (0.0, 0.2, 0.05, 0.0)[:nmat], (1.0, 2.0, 4.0, 0.5)[:nmat]
    pd = mat_problem(pd, gam, pinf)
    st = sale.State(md, pd)
    o = oracle.Oracle.from_problem(md, pd)
    rng = np.random.default_rng(2209)
    w = rng.random((nmat, md.ncell)) * (rng.random((nmat, md.ncell)) > 0.3) + 1e-3
    alpha = w / w.sum(axis=0)
    vol = o.field("vol")
    # one pressure in every material of a cell: 0.5 in the 3x3x3 corner block, 1e-3 elsewhere
    cell = np.arange(md.ncell)
    i, j, k3 = cell % md.nx, (cell // md.nx) % md.ny, cell // (md.nx * md.ny)
    p = np.where((i < 3) & (j < 3) & (k3 < 3), 0.5, 1e-3)
    mm = [alpha[k] * rho[k] * vol for k in range(nmat)]
    me = [(p + gam[k] * pinf[k]) / ((gam[k] - 1.0) * rho[k]) for k in range(nmat)]
    assert o.set_materials(list(alpha), mm, me) == 0
    for k in range(nmat):
        st.set_field(f"alpha{k}", alpha[k])
        st.set_field(f"m{k}", mm[k])
        st.set_field(f"e{k}", me[k])
    # node masses of the new cell masses (an eighth of each cell's)
    nx, ny, nz = md.nx, md.ny, md.nz
    mc = o.field("m").reshape(nz, ny, nx) / 8.0
    mn = np.zeros((nz + 1, ny + 1, nx + 1))
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                mn[dk:dk + nz, dj:dj + ny, di:di + nx] += mc
    mn = mn.reshape(-1)
    st.set_field("mn", mn)
    st.refresh()
    zero = np.zeros(md.nnode)
    assert o.set_state(o.field("x"), o.field("y"), o.field("z"), zero, zero, zero, mn, o.field("m"),
                       o.field("e"), t=o.s.t, dt_last=o.s.dt_last) == 0
    compare(st, o, tol=1e-13)
    assert st.diagnostics()["dt"] == pytest.approx(o.s.dt, rel=1e-12)
    assert st.run_to_time(max_cycles=30, remap_every=1) == 30
    rc, n = o.run(max_cycles=30, remap_every=1)
    assert rc == 0 and n == 30
    compare(st, o)
    compare_materials(st, o, nmat)


def test_identical_materials_equal_one_gas_on_the_gpu(sale):
    md = inputs.MeshDesc(20, 18, 16, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    one = sale.State(md, pd)
    two = sale.State(md, mat_problem(pd, (1.4, 1.4), (0.0, 0.0)))
    for st in (one, two):
        assert st.run_to_time(max_cycles=60, remap_every=1) == 60
    for f in NODE_FIELDS + CELL_FIELDS:
        a, b = two.field(f), one.field(f)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), f


def test_two_material_conservation(sale):
    md = inputs.MeshDesc(24, 24, 24, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=0.1)
    _, pd = inputs.sedov_octant(8)
    st = sale.State(md, mat_problem(pd, (1.4, 3.0), (0.0, 1e-6), x_split=0.25))
    d0 = st.diagnostics()
    mats0 = [st.field("m0").sum(), st.field("m1").sum()]
    assert st.run_to_time(max_cycles=100, remap_every=1) == 100
    d1 = st.diagnostics()
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-13)
    assert abs(d1["etot"] - d0["etot"]) <= 1e-12 * abs(d0["etot"])
    for m_now, m_start in zip([st.field("m0").sum(), st.field("m1").sum()], mats0):
        assert m_now == pytest.approx(m_start, rel=1e-7)
    a0, a1 = st.field("alpha0"), st.field("alpha1")
    assert np.max(np.abs(a0 + a1 - 1.0)) <= 1e-15
    assert np.sum((a1 > 0.0) & (a1 < 1.0)) > 0


def test_material_rules(sale):
    import ctypes as C
    md, pd = inputs.sod_x(20, 4, 4)
    pm = mat_problem(pd, (1.4, 3.0), (0.0, 0.5))
    m = sale.Mesh(md)
    base = sale.sale_state_bytes(m._h, sale.SALE_FP64)
    need = sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(pm)), sale.SALE_FP64)
    assert need >= base + (3 + 9) * 2 * 8 * md.ncell
    for bad, prec in ((pm, sale.SALE_FP32_MIXED), (dataclasses.replace(pm, remap_order=2), sale.SALE_FP64),
                      (dataclasses.replace(pm, shear0=1.0), sale.SALE_FP64),
                      (dataclasses.replace(pm, nmat=5), sale.SALE_FP64),
                      (dataclasses.replace(pm, mat_gamma=(1.0, 3.0, 1.4, 1.4)), sale.SALE_FP64),
                      (dataclasses.replace(pm, mat_pinf=(0.0, -1.0, 0.0, 0.0)), sale.SALE_FP64)):
        with pytest.raises(sale.SaleError) as ei:
            sale.State(md, bad, precision=prec)
        assert ei.value.code == sale.SALE_EINVAL
    st = sale.State(md, pm)
    with pytest.raises(sale.SaleError):  # the cell totals derive from the materials
        st.set_field("m", st.field("m"))
    with pytest.raises(sale.SaleError):  # material 2 does not exist
        st.field("alpha2")
    one = sale.State(md, pd)
    with pytest.raises(sale.SaleError):  # no materials on a single-gas state
        one.field("alpha0")
    with pytest.raises(sale.SaleError) as ei:  # batches run one material
        sale.Batch([(md, pm)])
    assert ei.value.code == sale.SALE_EINVAL
