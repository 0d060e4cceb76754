"""Batched runs: many independent meshes advanced by replays of captured graphs.

Each mesh of a batch must come out bitwise equal to the same mesh advanced
on its own (same precision, same kernels), whatever its size, problem and
time step; the batch API rejects what it does not run.
"""
import numpy as np
import pytest

from paper_2209_01983_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def small_instances(count=7):
    inst = inputs.batch_instances(count, seed=77, nmin=5, nmax=19)
    md, pd = inputs.sedov_octant(9, jitter=0.1)
    inst.append((md, pd))  # one jittered mesh with a point energy deposit
    return inst


FIELDS = ("m", "e", "rho", "u", "v", "w", "mn")


# (64 + 9): a replayed 64-cycle graph then a 9-cycle one; (131, 3): two
# replays, an odd tail, then a run that starts from swapped velocity roles
@pytest.mark.parametrize("runs", [(30,), (7, 8), (73,), (131, 3)])
def test_batch_matches_single_meshes_bitwise(sale, runs):
    inst = small_instances()
    b = sale.Batch(inst)
    for r in runs:
        assert b.run(r) == r
    total = sum(runs)
    ts = set()
    for i, (md, pd) in enumerate(inst):
        alone = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
        assert alone.run_to_time(max_cycles=total, remap_every=1) == total
        mine = b.state(i)
        for f in FIELDS:
            assert np.array_equal(mine.field(f), alone.field(f)), (i, f)
        d_b, d_a = mine.diagnostics(), alone.diagnostics()
        assert d_b["t"] == d_a["t"] and d_b["cycle"] == d_a["cycle"] == total
        ts.add(d_b["t"])
    assert len(ts) > 1  # every mesh took its own time steps


def test_batch_mesh_can_also_run_alone(sale):
    inst = small_instances(3)
    b = sale.Batch(inst)
    b.run(4)
    b.state(1).run_to_time(max_cycles=3, remap_every=1)  # one mesh advanced on its own
    b.run(5)
    for i, (md, pd) in enumerate(inst):
        alone = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
        alone.run_to_time(max_cycles=12 if i == 1 else 9, remap_every=1)
        assert np.array_equal(b.state(i).field("e"), alone.field("e")), i


def test_batch_api_checks(sale):
    import ctypes as C
    md = inputs.MeshDesc(4, 4, 4)
    descs = (sale.sale_mesh_desc * 1)(sale.mesh_desc(md))
    assert sale.sale_batch_bytes(1, descs, sale.SALE_FP64) == 0
    assert sale.sale_batch_bytes(0, descs, sale.SALE_FP32_MIXED) == 0
    b = sale.Batch(small_instances(2))
    with pytest.raises(sale.SaleError) as ei:
        sale.check(sale.sale_batch_run(b._h, 3, 0, None))
    assert ei.value.code == sale.SALE_EINVAL
    assert sale.sale_batch_state(b._h, 5) is None
