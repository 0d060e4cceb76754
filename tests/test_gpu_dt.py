"""The GPU time step against closed forms, through the C ABI.

The same cases that pin the oracle's step control (reading R5; see
test_oracle_dt.py for the derivations): a gas at rest on a box with three
different spacings (dt = cfl min(dx, dy, dz) / sqrt(gamma p / rho)); the
affine compression u = -alpha (x - 1/2) (div u = -3 alpha, L = h, so
dt = cfl h / sqrt(cs^2 + 2 q / rho) with q = rho (c_q (L div)^2 + c_l cs L
|div|)); a cell with negative energy (no sound speed); the exact growth
factor after a capped first step.  FP64 states to 1e-13, FP32-mixed ones to
FP32 rounding (the mixed step is evaluated in FP32).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def tol(sale, prec):
    return 1e-13 if prec == sale.SALE_FP64 else 2e-6


@pytest.mark.parametrize("mixed", [False, True])
def test_rest_box_dt(sale, mixed):
    prec = sale.SALE_FP32_MIXED if mixed else sale.SALE_FP64
    md = inputs.MeshDesc(6, 5, 4, lo=(0.0, 0.0, 0.0), hi=(0.6, 1.0, 0.2))
    for rho, p, gamma, cfl in ((1.3, 0.7, 1.4, 0.3), (0.2, 5.0, 1.67, 0.45)):
        pd = inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=rho, p_bg=p, gamma=gamma, cfl=cfl)
        st = sale.State(md, pd, precision=prec)
        want = cfl * 0.05 / math.sqrt(gamma * p / rho)
        dt = st.diagnostics()["dt"]
        assert abs(dt - want) <= tol(sale, prec) * want, (dt, want)
        st.run_to_time(max_cycles=3, remap_every=1)
        dt = st.diagnostics()["dt"]
        assert abs(dt - want) <= tol(sale, prec) * want, (dt, want)


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("alpha,c_q,c_l", [(2.0, 1.0, 0.5), (2.0, 1.0, 0.0), (2.0, 0.0, 0.5), (-2.0, 1.0, 0.5)])
def test_affine_compression_dt(sale, mixed, alpha, c_q, c_l):
    prec = sale.SALE_FP32_MIXED if mixed else sale.SALE_FP64
    md = inputs.MeshDesc(4, 4, 4)
    pd = inputs.ProblemDesc(kind=inputs.PROB_UNIFORM, rho_bg=1.0, p_bg=1.0, gamma=1.4, c_q=c_q, c_l=c_l)
    st = sale.State(md, pd, precision=prec)
    x, y, z = st.mesh.nodes()
    for name, c in (("u", x), ("v", y), ("w", z)):
        st.set_field(name, -alpha * (c - 0.5))
    st.refresh()
    cs2, ldiv = 1.4, 3.0 * alpha * 0.25
    q = (c_q * ldiv * ldiv + c_l * math.sqrt(cs2) * ldiv) if alpha > 0 else 0.0
    want = 0.3 * 0.25 / math.sqrt(cs2 + 2.0 * q)
    dt = st.diagnostics()["dt"]
    assert abs(dt - want) <= tol(sale, prec) * want * 4, (dt, want)
    got_q = st.field("q")
    if q == 0.0:
        assert np.all(got_q == 0.0)
    else:
        assert np.max(np.abs(got_q - q)) <= tol(sale, prec) * 8 * q
    # and the oracle, given the same velocities, agrees
    o = oracle.Oracle.from_problem(md, pd)
    rc = o.set_state(o.field("x"), o.field("y"), o.field("z"), -alpha * (x - 0.5), -alpha * (y - 0.5),
                     -alpha * (z - 0.5), o.field("mn"), o.field("m"), o.field("e"))
    assert rc == 0
    assert abs(o.s.dt - want) <= 1e-13 * want


def test_negative_energy_cell_fp64(sale):
    md, pd = inputs.uniform_box(4, rho=1.0, p=1.0)
    st = sale.State(md, pd)
    e = st.field("e")
    e[5] = -1e-3
    st.set_field("e", e)
    st.refresh()
    d = st.diagnostics()
    assert d["status"] == 0
    assert st.field("cs")[5] == 0.0
    want = 0.3 * 0.25 / math.sqrt(1.4)
    assert abs(d["dt"] - want) <= 1e-13 * want


@pytest.mark.parametrize("mixed", [False, True])
def test_first_step_cap_then_exact_growth(sale, mixed):
    prec = sale.SALE_FP32_MIXED if mixed else sale.SALE_FP64
    md, pd = inputs.sedov_octant(12)
    pd.dt_init = 1e-7
    st = sale.State(md, pd, precision=prec)
    assert st.diagnostics()["dt"] == 1e-7
    dt = 1e-7
    for _ in range(5):
        st.run_to_time(max_cycles=1, remap_every=1)
        nxt = st.diagnostics()["dt"]
        assert nxt == 1.1 * dt, (nxt, dt)
        dt = nxt
