"""Degenerate meshes through every path: a single cell, one-cell-thick
slabs and lines (every node on a wall, tiles that are all tail).

FP64 against the oracle at 1e-10 (Lagrange and Eulerian cycles, with and
without the scheme options); FP32-mixed against FP64 (L1 <= 1e-4); a batch
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
