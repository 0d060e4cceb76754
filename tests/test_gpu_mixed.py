"""FP32-mixed Eulerian path against the FP64 GPU path (which is held to the
oracle by test_gpu_parity.py), through the C ABI.

Bar: relative L1 error of density and specific internal energy
sum|a - b| V / sum|b| V <= 1e-4 against FP64 on the same mesh and the same
number of cycles; the conservation drift of the mixed run is reported and
bounded.
"""
import numpy as np
import pytest

from paper_2209_01983_gb300 import inputs

pytestmark = pytest.mark.gpu

L1_TOL = 1e-4


@pytest.fixture(scope="module")
def sale():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale as s
    return s


def l1_rel(a, b, w):
    return float(np.sum(np.abs(a - b) * w) / np.sum(np.abs(b) * w))


@pytest.mark.parametrize("n,jitter,cycles", [(32, 0.0, 150), (30, 0.1, 150), (48, 0.1, 60)])
def test_mixed_matches_fp64(sale, n, jitter, cycles):
    md, pd = inputs.sedov_octant(n, jitter=jitter)
    s64 = sale.State(md, pd, precision=sale.SALE_FP64)
    s32 = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    d0 = s32.diagnostics()
    assert s64.run_to_time(max_cycles=cycles, remap_every=1) == cycles
    assert s32.run_to_time(max_cycles=cycles, remap_every=1) == cycles
    w = s64.field("vol")
    errs = {f: l1_rel(s32.field(f), s64.field(f), w) for f in ("rho", "e")}
    assert all(v <= L1_TOL for v in errs.values()), errs
    d64, d32 = s64.diagnostics(), s32.diagnostics()
    # the two runs took the same steps (dt agrees to FP32 accuracy)
    assert abs(d32["t"] - d64["t"]) <= 1e-5 * d64["t"]
    # conservation drift of the mixed run (FP64 sums of FP32 fields)
    assert abs(d32["mass"] - d0["mass"]) <= 1e-5 * d0["mass"]
    assert abs(d32["etot"] - d0["etot"]) <= 1e-4 * d0["etot"]
    assert d32["ke"] > 1e-3 * d0["etot"]


def test_mixed_uniform_state_at_rest(sale):
    md, pd = inputs.uniform_box(12, rho=1.0, p=1.0, jitter=0.1, seed=4)
    st = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    e0 = st.field("e")
    st.run_to_time(max_cycles=20, remap_every=1)
    # uniform p+q: the face terms cancel; what is left comes from FP32
    # rounding of m and V_E (rho = m / V_E differs by an ulp between cells)
    cs = float(np.sqrt(1.4 * 0.4 * e0.max()))
    for f in "uvw":
        assert np.max(np.abs(st.field(f))) <= 1e-6 * cs
    assert np.max(np.abs(st.field("e") - e0) / e0) <= 1e-6


def test_mixed_deterministic(sale):
    md, pd = inputs.sedov_octant(20, jitter=0.1)
    outs = []
    for _ in range(2):
        st = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
        st.run_to_time(max_cycles=25, remap_every=1)
        outs.append([st.field(f) for f in ("e", "u", "mn")])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_mixed_state_api(sale):
    md, pd = inputs.sedov_octant(10)
    st = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    for call in (lambda: st.lagrange_step(), lambda: st.remap_step(),
                 lambda: st.run_to_time(max_cycles=2, remap_every=0)):
        with pytest.raises(sale.SaleError) as ei:
            call()
        assert ei.value.code == sale.SALE_ESTATE
    st.run_to_time(max_cycles=3, remap_every=1)
    rho, p, e = st.field("rho"), st.field("p"), st.field("e")
    assert np.allclose(p, 0.4 * rho * e, rtol=1e-6, atol=0)
    assert np.array_equal(st.field("x"), st.field("xref"))
    assert st.field("vol").min() > 0


def test_mixed_node_mass_stays_consistent(sale):
    # m_n = sum of the adjacent cell masses / 8 holds exactly in exact
    # arithmetic (the dual-mesh fluxes are built from the cell fluxes); the
    # float-float node mass keeps the FP32 run within a few ulps per cycle
    # of it (a plain FP32 node mass drifted by ~1e-3 over such a run)
    n = 72
    md, pd = inputs.sedov_octant(n, jitter=0.1)
    st = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    assert st.run_to_time(max_cycles=900, remap_every=1) == 900
    mc = st.field("m").reshape(n, n, n)
    p = np.zeros((n + 2, n + 2, n + 2))
    p[1:-1, 1:-1, 1:-1] = mc
    want = sum(p[dk:dk + n + 1, dj:dj + n + 1, di:di + n + 1]
               for dk in (0, 1) for dj in (0, 1) for di in (0, 1)).ravel() / 8.0
    mn = st.field("mn")
    assert float(np.max(np.abs(mn - want) / want)) <= 5e-5


def test_mixed_field_transfer_roundings(sale):
    # FP32-mixed fields take FP64 input as hi = fl32(x) (plus lo = fl32(x - hi)
    # for the float-float m, e and m_n) and read back as hi (+ lo) in FP64,
    # converted on the device: exactly the host formulas, at any size
    md, pd = inputs.sedov_octant(11, jitter=0.1)
    st = sale.State(md, pd, precision=sale.SALE_FP32_MIXED)
    st.run_to_time(max_cycles=3, remap_every=1)
    rng = np.random.default_rng(5)

    def hi(x):
        return x.astype(np.float32).astype(np.float64)

    for name, ff in (("e", True), ("m", True), ("mn", True), ("u", False), ("w", False)):
        x = st.field(name) * (1.0 + 1e-3 * rng.uniform(-1, 1, st.field(name).size)) + 1e-9
        st.set_field(name, x)
        want = hi(x) + hi(x - hi(x)) if ff else hi(x)
        assert np.array_equal(st.field(name), want), name
        if ff:
            assert float(np.max(np.abs(st.field(name) - x) / np.abs(x))) <= 2.0 ** -45
    st.refresh()
    rho, p, e = st.field("rho"), st.field("p"), st.field("e")
    assert np.allclose(p, 0.4 * rho * e, rtol=1e-6, atol=0)
    assert st.run_to_time(max_cycles=3, remap_every=1) == 3
