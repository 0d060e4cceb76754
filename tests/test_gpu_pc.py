"""Predictor-corrector Lagrangian step (time_order = 2) on the GPU.

FP64 paths against the oracle's predictor-corrector: relative L-infinity
<= 1e-10 per field.  FP32-mixed against the FP64 GPU run with the same
step: relative L1 of density and energy <= 1e-4.  Total energy exact to
roundoff on the FP64 path; the sizing and batch rules of the option.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def pc(pd, **kw):
    return dataclasses.replace(pd, time_order=2, **kw)


def test_sod_lagrange_matches_oracle(sale):
    md, pd = inputs.sod_x(100, 4, 4)
    pd = pc(pd)
    st = sale.State(md, pd)
    d0 = st.diagnostics()
    n = st.run_to_time(t_end=0.2)
    o = oracle.Oracle.from_problem(md, pd)
    rc, n_o = o.run(t_end=0.2)
    assert rc == 0 and n == n_o
    compare(st, o)
    d = st.diagnostics()
    assert abs(d["etot"] - d0["etot"]) <= 1e-13 * d0["etot"]


@pytest.mark.parametrize("dims,jitter,remap_every", [((23, 17, 14), 0.0, 1), ((16, 19, 13), 0.1, 1),
                                                     ((14, 12, 10), 0.05, 3), ((12, 11, 10), 0.1, 0)])
def test_sedov_matches_oracle(sale, dims, jitter, remap_every):
    md, pd = inputs.sedov_octant(1, jitter=jitter)
    md.nx, md.ny, md.nz = dims
    pd = pc(pd)
    cycles = 100 if remap_every == 1 else 40
    st = sale.State(md, pd)
    assert st.run_to_time(max_cycles=cycles, remap_every=remap_every) == cycles
    o = oracle.Oracle.from_problem(md, pd)
    rc, n_o = o.run(max_cycles=cycles, remap_every=remap_every)
    assert rc == 0 and n_o == cycles
    compare(st, o)


def test_explicit_steps_match_oracle(sale):
    md, pd = inputs.sedov_octant(10, jitter=0.1)
    pd = pc(pd, remap_order=2)
    st = sale.State(md, pd)
    o = oracle.Oracle.from_problem(md, pd)
    for it in range(5):
        dt = 1e-4 * (1 + it)
        st.lagrange_step(dt)
        o.check(o.lagrange_step(dt))
        if it % 2:
            st.remap_step()
            o.check(o.remap_step())
    compare(st, o)


def test_pc_differs_from_single_stage(sale):
    md, pd = inputs.sedov_octant(12, jitter=0.1)
    a, b = sale.State(md, pd), sale.State(md, pc(pd))
    a.run_to_time(max_cycles=30, remap_every=1)
    b.run_to_time(max_cycles=30, remap_every=1)
    assert np.max(np.abs(a.field("e") - b.field("e"))) > 1e-6 * np.max(a.field("e"))


@pytest.mark.parametrize("n,jitter,cycles", [(32, 0.0, 120), (30, 0.1, 120)])
def test_mixed_matches_fp64(sale, n, jitter, cycles):
    md, pd = inputs.sedov_octant(n, jitter=jitter)
    pd = pc(pd)
    s64 = sale.State(md, pd, precision=sale.SALE_FP64)
    s32 = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    d0 = s32.diagnostics()
    assert s64.run_to_time(max_cycles=cycles, remap_every=1) == cycles
    assert s32.run_to_time(max_cycles=cycles, remap_every=1) == cycles
    w = s64.field("vol")
    for f in ("rho", "e"):
        a, b = s32.field(f), s64.field(f)
        assert float(np.sum(np.abs(a - b) * w) / np.sum(np.abs(b) * w)) <= 1e-4, f
    d32 = s32.diagnostics()
    assert abs(d32["mass"] - d0["mass"]) <= 1e-5 * d0["mass"]
    assert abs(d32["etot"] - d0["etot"]) <= 1e-4 * d0["etot"]


def test_mixed_uniform_state_at_rest(sale):
    md, pd = inputs.uniform_box(12, rho=1.0, p=1.0, jitter=0.1, seed=4)
    st = sale.State(md, pc(pd), precision=sale.SALE_FP32_MIXED)
    st.run_to_time(max_cycles=20, remap_every=1)
    for f in "uvw":
        assert float(np.max(np.abs(st.field(f)))) <= 1e-6


def test_sizing_and_batch_rules(sale):
    import ctypes as C
    md, pd = inputs.sedov_octant(8)
    m = sale.Mesh(md)
    base = sale.sale_state_bytes(m._h, sale.SALE_FP64)
    need = sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(pc(pd))), sale.SALE_FP64)
    assert need > base
    import torch
    buf = torch.empty(base, dtype=torch.uint8, device="cuda")
    h = sale._vp()
    rc = sale.sale_state_init(m._h, C.byref(sale.problem_desc(pc(pd))), sale.SALE_FP64, sale._vp(buf.data_ptr()),
                              base, None, C.byref(h))
    assert rc == sale.SALE_ENOMEM  # the buffer is smaller than the option needs
    with pytest.raises(sale.SaleError) as ei:
        sale.Batch([(md, pc(pd))])
    assert ei.value.code == sale.SALE_EINVAL
