"""Material strength (the stress module) on the GPU: FP64 against the
oracle, element by element, through the C ABI.

The deviatoric stress components are compared normwise over the six of
them (like the velocity components), the plastic strain on its own scale;
tolerance 1e-10 relative L-infinity as for every other FP64 field.  The
oracle side of each case is pinned in test_oracle_strength.py.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs
from test_gpu_parity import CELL_FIELDS, NODE_FIELDS, compare
import test_gpu_parity

pytestmark = pytest.mark.gpu

STRESS = ("sxx", "syy", "szz", "sxy", "syz", "szx")
for _f in STRESS:
    test_gpu_parity.GROUPS[_f] = STRESS
FIELDS = NODE_FIELDS + CELL_FIELDS + STRESS + ("eps_p",)

# an elastic-plastic material for the Sedov blast (background p = 1e-6):
# the blast region yields and work-hardens, the rest stays elastic
SEDOV_STRENGTH = dict(shear0=0.05, shear_dp=0.3, shear_dt=-0.01, cv=1.0, e_ref=0.0, rho_ref=1.0, yield0=2e-3,
                      yield_max=1e-2, hard_beta=20.0, hard_n=0.3)


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def sedov(n=(15, 13, 11), jitter=0.1, **extra):
    md = inputs.MeshDesc(*n, lo=(0.0, 0.0, 0.0), hi=(1.2, 1.2, 1.2), jitter=jitter)
    _, pd = inputs.sedov_octant(8)
    pd = dataclasses.replace(pd, **dict(SEDOV_STRENGTH, **extra))
    return md, pd


@pytest.mark.parametrize("remap_every,cycles", [(0, 60), (1, 40), (3, 45)])
def test_strength_sedov_against_oracle(sale, remap_every, cycles):
    md, pd = sedov()
    st = sale.State(md, pd)
    assert st.run_to_time(max_cycles=cycles, remap_every=remap_every) == cycles
    o = oracle.Oracle.from_problem(md, pd)
    rc, n = o.run(max_cycles=cycles, remap_every=remap_every)
    assert rc == 0 and n == cycles
    assert np.any(o.field("eps_p") > 0.0)  # the material yielded
    compare(st, o, fields=FIELDS)
    d = st.diagnostics()
    assert d["dt"] == pytest.approx(o.s.dt, rel=1e-10)


def test_strength_second_order_remap_and_hourglass(sale):
    md, pd = sedov(remap_order=2, c_hg=0.05)
    st = sale.State(md, pd)
    assert st.run_to_time(max_cycles=30, remap_every=1) == 30
    o = oracle.Oracle.from_problem(md, pd)
    rc, n = o.run(max_cycles=30, remap_every=1)
    assert rc == 0 and n == 30
    compare(st, o, fields=FIELDS)


def test_elastic_bar_against_oracle(sale):
    # the bar of the oracle's wave-period pin at a larger amplitude: each
    # node force is the difference of two O(1) pressures, so a wave of
    # amplitude eps carries rounding of ~1e-16 / (eps pi h) a step, and the
    # stress integrates a velocity gradient that cancels ~30-fold more (on
    # the oracle alone, a last-bit change of e moves s_xx by 2e-10 at
    # eps = 1e-4 and by 5e-12 at eps = 1e-2 over 40 cycles)
    nx = 100
    md = inputs.MeshDesc(nx, 1, 1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0 / nx, 1.0 / nx))
    pd = inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=1.0, p_bg=1.0, gamma=1.4,
                            shear0=3.0, cv=1.0, rho_ref=1.0, yield0=1e30, yield_max=1e30)
    st = sale.State(md, pd)
    o = oracle.Oracle.from_problem(md, pd)
    x, y, z = st.mesh.nodes()
    u = 1e-2 * np.sin(math.pi * x)
    st.set_field("u", u)
    st.refresh()
    zero = np.zeros_like(u)
    assert o.set_state(o.field("x"), o.field("y"), o.field("z"), u, zero, zero, o.field("mn"), o.field("m"),
                       o.field("e")) == 0
    assert st.diagnostics()["dt"] == pytest.approx(o.s.dt, rel=1e-12)
    assert st.run_to_time(max_cycles=40) == 40
    rc, n = o.run(max_cycles=40)
    assert rc == 0 and n == 40
    compare(st, o, fields=("x", "u", "m", "e", "rho", "p", "sxx", "syy", "szz"))


def test_zero_yield_is_bitwise_hydro_on_the_gpu(sale):
    md, pd = sedov(n=(12, 12, 12), yield0=0.0)
    hydro = dataclasses.replace(pd, shear0=0.0)
    a, b = sale.State(md, hydro), sale.State(md, pd)
    dt = 0.5 * a.diagnostics()["dt"]
    for n in range(12):
        a.lagrange_step(dt)
        b.lagrange_step(dt)
        if n % 3 == 2:
            a.remap_step()
            b.remap_step()
    for f in NODE_FIELDS + ("m", "e", "p", "q"):
        assert np.array_equal(a.field(f), b.field(f)), f
    for f in STRESS:
        assert np.all(b.field(f) == 0.0), f


def test_strength_energy_exact(sale):
    md, pd = sedov(n=(20, 20, 20))
    st = sale.State(md, pd)
    d0 = st.diagnostics()
    assert st.run_to_time(max_cycles=80, remap_every=1) == 80
    d1 = st.diagnostics()
    assert abs(d1["etot"] - d0["etot"]) <= 1e-12 * abs(d0["etot"])
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-13)


def test_strength_rules(sale):
    import ctypes as C
    md, pd = sedov(n=(8, 8, 8))
    m = sale.Mesh(md)
    base = sale.sale_state_bytes(m._h, sale.SALE_FP64)
    need = sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(pd)), sale.SALE_FP64)
    assert need >= base + (9 + 7) * 8 * md.ncell  # stress, plastic strain, G, Y; the remap copy
    with pytest.raises(sale.SaleError) as ei:
        sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    assert ei.value.code == sale.SALE_EINVAL
    with pytest.raises(sale.SaleError) as ei:
        sale.State(md, dataclasses.replace(pd, time_order=2))
    assert ei.value.code == sale.SALE_EINVAL
    with pytest.raises(sale.SaleError) as ei:
        sale.State(md, dataclasses.replace(pd, cv=0.0))
    assert ei.value.code == sale.SALE_EINVAL
