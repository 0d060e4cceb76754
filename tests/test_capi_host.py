"""Host-side checks of the C ABI library (no GPU needed).

The library must load, export every function include/sale.h declares, and
its host-only calls (mesh generation, sizing, argument validation) must
behave; the mesh generator must agree bit for bit with the seeded inputs
module, since the oracle receives the inputs module's mesh.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2209_01983_gb300 import inputs


@pytest.fixture(scope="module")
def sale():
    from paper_2209_01983_gb300 import build
    build.build()
    from paper_2209_01983_gb300 import sale as s
    return s


def header_functions():
    text = open(os.path.join(ROOT, "include", "sale.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sale_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(sale):
    names = header_functions()
    assert len(names) >= 15
    lib = C.CDLL(sale.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sale.EXPORTS)


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_mesh_matches_inputs_module_bitwise(sale, jitter):
    md = inputs.MeshDesc(7, 5, 6, lo=(0.0, -0.3, 1.0), hi=(1.2, 0.9, 1.7), jitter=jitter, seed=2209)
    got = sale.Mesh(md).nodes()
    want = inputs.mesh_nodes(md)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_mesh_validation(sale):
    bad = [inputs.MeshDesc(0, 4, 4), inputs.MeshDesc(4, 4, 4, jitter=0.6),
           inputs.MeshDesc(4, 4, 4, lo=(1.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)),
           inputs.MeshDesc(4, 4, 4, reflect=(1, 1, 1, 1, 1, 0))]
    for md in bad:
        with pytest.raises(sale.SaleError) as ei:
            sale.Mesh(md)
        assert ei.value.code == sale.SALE_EINVAL


def test_state_bytes(sale):
    md = inputs.MeshDesc(8, 8, 8)
    m = sale.Mesh(md)
    b64 = sale.sale_state_bytes(m._h, sale.SALE_FP64)
    assert b64 >= 8 * (17 * md.nnode + 14 * md.ncell)
    assert sale.sale_state_bytes(m._h, 7) == 0


def test_null_arguments_rejected(sale):
    assert sale.sale_mesh_create(None, None) == sale.SALE_EINVAL
    assert sale.sale_lagrange_step(None, 0.0) == sale.SALE_EINVAL
    assert sale.sale_run_to_time(None, 1.0, 1, 0, None) == sale.SALE_EINVAL
    assert b"null" in sale.sale_last_error()


def test_state_bytes_for_scheme_options(sale):
    import dataclasses
    md, pd = inputs.sedov_octant(8, jitter=0.1)
    m = sale.Mesh(md)
    for prec in (sale.SALE_FP64, sale.SALE_FP32_MIXED):
        base = sale.sale_state_bytes(m._h, prec)
        assert sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(pd)), prec) == base
        pc = dataclasses.replace(pd, time_order=2)
        # half-step corner gradients: 24 values per cell
        extra = sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(pc)), prec) - base
        assert extra >= 24 * md.ncell * (8 if prec == sale.SALE_FP64 else 4)
    o2 = dataclasses.replace(pd, remap_order=2)
    assert sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(o2)), sale.SALE_FP64) >= \
        sale.sale_state_bytes(m._h, sale.SALE_FP64) + 7 * 8 * md.ncell
    assert sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(o2)), sale.SALE_FP32_MIXED) == \
        sale.sale_state_bytes(m._h, sale.SALE_FP32_MIXED)
    assert sale.sale_state_bytes_for(m._h, None, sale.SALE_FP64) == 0
    # hourglass corner forces: 24 values per cell; FP64 also caches the 32
    # projected shape vectors of every reference cell
    hg = dataclasses.replace(pd, c_hg=0.1)
    for prec, per_cell in ((sale.SALE_FP64, (24 + 32) * 8), (sale.SALE_FP32_MIXED, 24 * 4)):
        assert sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(hg)), prec) >= \
            sale.sale_state_bytes(m._h, prec) + per_cell * md.ncell


def test_state_bytes_for_materials(sale):
    import dataclasses
    md, pd = inputs.sedov_octant(8, jitter=0.1)
    m = sale.Mesh(md)
    base = sale.sale_state_bytes(m._h, sale.SALE_FP64)
    for nmat in (2, 3, 4):
        pm = dataclasses.replace(pd, nmat=nmat)
        # fraction, mass, energy of every material; its volume, mass and
        # energy fluxes through the three low faces
        got = sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(pm)), sale.SALE_FP64)
        assert got >= base + (3 + 9) * nmat * 8 * md.ncell
    # one material is the plain state; FP32-mixed states take no materials
    assert sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(dataclasses.replace(pd, nmat=1))),
                                     sale.SALE_FP64) == base
    assert sale.sale_state_bytes_for(m._h, C.byref(sale.problem_desc(dataclasses.replace(pd, nmat=2))),
                                     sale.SALE_FP32_MIXED) == sale.sale_state_bytes(m._h, sale.SALE_FP32_MIXED)
