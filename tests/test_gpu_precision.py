"""FP32-mixed against FP64 on the precision workload and on thin cells.

The precision workload is the Sedov octant run to t = 0.5 with the Eulerian
remap every cycle; here at 96^3 cells (the workload's 256^3 runs in
bench.py --config precision).  The error measure is the relative L1 norm of
the mixed run's density and specific internal energy against the FP64 run
on the same mesh, weighted by the FP64 cell volume (and, for e, also by the
cell mass and outside the near-vacuum core, rho < 1e-3 of its maximum).
The bounds asserted below, with the values measured on GB300 (the GPU
arithmetic is deterministic):

    96^3, t = 0.5 (2148 cycles)   measured   bound
    L1(rho), volume-weighted      3.9e-8     1e-6
    L1(e), mass-weighted          5.0e-6     1e-4
    L1(e), outside the core       2.9e-5     1e-4
    L1(e), volume-weighted        1.46e-4    5e-4
    total-energy drift (mixed)    7.7e-9     1e-7

The volume-weighted L1(e) is the one measure above 1e-4: the near-vacuum
core (0.3% of the volume) holds e = E/m of cells with almost no mass, where
FP32 roundings of the nearly uniform pressure feed the force differences;
it grows with resolution (7.5e-7 at 64^3, 1.46e-4 at 96^3, 4.1e-4 at
128^3).

Thin cells: a Sod tube of 100 x 4 x 4 cells on [0, 1] x [0, 2e-4]^2 (aspect
200), Eulerian every cycle to t = 0.2 (about 16,600 cycles, the CFL step
set by the thin direction), plain and jittered: L1(rho) 6.5e-5 / 7.8e-5 and
L1(e) 2.0e-5 / 2.4e-5, asserted <= 1e-4.  The FP64 path stays within 1e-10
of the oracle on the same thin cells.
"""
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


def l1(a, b, w):
    return float(np.sum(np.abs(a - b) * w) / np.sum(np.abs(b) * w))


def fields(st):
    return {f: st.field(f) for f in ("m", "e", "rho", "vol")}


def test_precision_workload_sedov96(sale):
    md, pd = inputs.sedov_octant(96)
    s32 = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    d0 = s32.diagnostics()
    c32 = s32.run_to_time(t_end=0.5, remap_every=1)
    d1 = s32.diagnostics()
    a = fields(s32)
    s32.close()
    s64 = sale.State(md, pd)
    c64 = s64.run_to_time(t_end=0.5, remap_every=1)
    b = fields(s64)
    s64.close()
    assert c32 == c64
    w, wm = b["vol"], b["m"]
    core = b["rho"] < 1e-3 * b["rho"].max()
    assert l1(a["rho"], b["rho"], w) <= 1e-6
    assert l1(a["e"], b["e"], wm) <= 1e-4
    assert l1(a["e"], b["e"], w * ~core) <= 1e-4
    assert l1(a["e"], b["e"], w) <= 5e-4
    assert float(np.sum(w * core) / np.sum(w)) <= 0.01  # the core is a small part of the volume
    assert abs(d1["etot"] - d0["etot"]) <= 1e-7 * abs(d0["etot"])
    assert d1["mass"] == d0["mass"] or abs(d1["mass"] - d0["mass"]) <= 1e-12 * d0["mass"]


def thin_tube(jitter):
    md, pd = inputs.sod_x(100, 4, 4)
    md.hi = (1.0, 2e-4, 2e-4)
    md.jitter = jitter
    return md, pd


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_thin_cells_mixed_against_fp64(sale, jitter):
    md, pd = thin_tube(jitter)
    s32 = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    s64 = sale.State(md, pd)
    c32 = s32.run_to_time(t_end=0.2, remap_every=1)
    c64 = s64.run_to_time(t_end=0.2, remap_every=1)
    assert c64 > 10000 and abs(c32 - c64) <= 1
    a, b = fields(s32), fields(s64)
    assert l1(a["rho"], b["rho"], b["vol"]) <= 1e-4
    assert l1(a["e"], b["e"], b["vol"]) <= 1e-4


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_thin_cells_fp64_against_oracle(sale, jitter):
    md, pd = thin_tube(jitter)
    st = sale.State(md, pd)
    assert st.run_to_time(max_cycles=100, remap_every=1) == 100
    o = oracle.Oracle.from_problem(md, pd)
    rc, n = o.run(max_cycles=100, remap_every=1)
    assert rc == 0 and n == 100
    compare(st, o)
