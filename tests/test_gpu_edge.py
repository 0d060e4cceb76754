"""Degenerate meshes through every path: a single cell, one-cell-thick
slabs and lines (every node on a wall, tiles that are all tail).

FP64 against the oracle at 1e-10 (Lagrange and Eulerian cycles, with and
without the scheme options, with strength and with two materials); FP32-mixed against FP64 (L1 <= 1e-4); a batch
of degenerate meshes bitwise against each mesh alone.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs
from test_gpu_parity import compare

pytestmark = pytest.mark.gpu

DIMS = [(1, 1, 1), (1, 7, 1), (9, 1, 1), (1, 1, 6), (2, 3, 1), (5, 1, 4)]


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def problem(dims, jitter=0.1):
    md, pd = inputs.sedov_octant(1, jitter=jitter)
    md.nx, md.ny, md.nz = dims
    md.hi = tuple(0.1 * d for d in dims)
    return md, pd


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("remap_every,opts", [(1, {}), (0, {}), (1, {"remap_order": 2, "time_order": 2, "c_hg": 0.05})])
def test_fp64_matches_oracle(sale, dims, remap_every, opts):
    md, pd = problem(dims)
    pd = dataclasses.replace(pd, **opts)
    st = sale.State(md, pd)
    assert st.run_to_time(max_cycles=25, remap_every=remap_every) == 25
    o = oracle.Oracle.from_problem(md, pd)
    rc, n = o.run(max_cycles=25, remap_every=remap_every)
    assert rc == 0 and n == 25
    compare(st, o)


STRENGTH = dict(shear0=0.05, shear_dp=0.3, shear_dt=-0.01, cv=1.0, rho_ref=1.0, yield0=2e-3, yield_max=1e-2,
                hard_beta=20.0, hard_n=0.3)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("remap_every,kind", [(1, "strength"), (0, "strength"), (1, "materials"), (0, "materials"),
                                              (3, "materials")])
def test_fp64_options_on_degenerate_meshes(sale, dims, remap_every, kind):
    from test_gpu_multimat import compare_materials
    md, pd = problem(dims)
    if kind == "strength":
        pd = dataclasses.replace(pd, **STRENGTH)
    else:  # material 1 from the middle of the box on (the whole box when it is one cell wide)
        pd = dataclasses.replace(pd, nmat=2, mat_gamma=(1.4, 3.0, 1.4, 1.4), mat_pinf=(0.0, 1e-6, 0.0, 0.0),
                                 x_split=0.05 * dims[0])
    st = sale.State(md, pd)
    assert st.run_to_time(max_cycles=25, remap_every=remap_every) == 25
    o = oracle.Oracle.from_problem(md, pd)
    rc, n = o.run(max_cycles=25, remap_every=remap_every)
    assert rc == 0 and n == 25
    compare(st, o)
    if kind == "materials":
        compare_materials(st, o, 2)
    else:  # the stress normwise over its six components, the plastic strain on its own scale
        comps = ("sxx", "syy", "szz", "sxy", "syz", "szx")
        scale = max(float(np.max(np.abs(o.field(f)))) for f in comps)
        for f in comps:
            assert float(np.max(np.abs(st.field(f) - o.field(f)))) <= 1e-10 * scale, f  # 0 on both: one cell
        ep = o.field("eps_p")
        assert float(np.max(np.abs(st.field("eps_p") - ep))) <= 1e-10 * float(np.max(ep))


@pytest.mark.parametrize("dims", DIMS)
def test_mixed_matches_fp64(sale, dims):
    md, pd = problem(dims)
    s64 = sale.State(md, pd, precision=sale.SALE_FP64)
    s32 = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    assert s64.run_to_time(max_cycles=25, remap_every=1) == 25
    assert s32.run_to_time(max_cycles=25, remap_every=1) == 25
    w = s64.field("vol")
    for f in ("rho", "e"):
        a, b = s32.field(f), s64.field(f)
        assert float(np.sum(np.abs(a - b) * w) / np.sum(np.abs(b) * w)) <= 1e-4, (dims, f)


def test_batch_of_degenerate_meshes_bitwise(sale):
    inst = [problem(d) for d in DIMS]
    b = sale.Batch(inst)
    assert b.run(12) == 12
    for i, (md, pd) in enumerate(inst):
        alone = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
        alone.run_to_time(max_cycles=12, remap_every=1)
        for f in ("m", "e", "u", "w"):
            assert np.array_equal(b.state(i).field(f), alone.field(f)), (i, f)
