"""Seeded synthetic inputs: generator definition, mesh jitter, problems."""
import os

import numpy as np

from conftest import ROOT
from paper_2209_01983_gb300 import inputs


def test_splitmix64_reference_sequence():
    want = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "splitmix64_seed0.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            want[k] = int(v, 16)
    got = inputs.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(g) for g in got] == [want["out0"], want["out1"], want["out2"]]


def test_uniform_mesh_and_jitter_bounds():
    md = inputs.MeshDesc(5, 4, 3, lo=(0.0, -1.0, 2.0), hi=(1.0, 1.0, 2.6), jitter=0.1, seed=9)
    x, y, z = inputs.mesh_nodes(md)
    flat = inputs.MeshDesc(5, 4, 3, lo=md.lo, hi=md.hi)
    x0, y0, z0 = inputs.mesh_nodes(flat)
    h = [(md.hi[d] - md.lo[d]) / n for d, n in enumerate((5, 4, 3))]
    kk, jj, ii = np.meshgrid(np.arange(4), np.arange(5), np.arange(6), indexing="ij")
    for d, (a, a0, idx, n) in enumerate(zip((x, y, z), (x0, y0, z0), (ii, jj, kk), (5, 4, 3))):
        off = (a - a0).reshape(idx.shape)
        assert np.all(np.abs(off) <= 0.1 * h[d] * (1 + 1e-12))
        wall = (idx == 0) | (idx == n)
        assert np.all(off[wall] == 0.0)
        assert np.count_nonzero(off[~wall]) == np.count_nonzero(~wall)
    # deterministic per seed, different across seeds
    assert np.array_equal(inputs.mesh_nodes(md)[0], x)
    md2 = inputs.MeshDesc(5, 4, 3, lo=md.lo, hi=md.hi, jitter=0.1, seed=10)
    assert not np.array_equal(inputs.mesh_nodes(md2)[0], x)


def test_sod_and_sedov_primitives():
    md, pd = inputs.sod_x(100, 4, 4)
    rho0, p0, dc, de = inputs.problem_prim(md, pd)
    r = rho0.reshape(4, 4, 100)
    assert np.all(r[:, :, :50] == 1.0) and np.all(r[:, :, 50:] == 0.125)
    assert dc == -1
    md, pd = inputs.sedov_octant(8)
    rho0, p0, dc, de = inputs.problem_prim(md, pd)
    assert dc == 0 and de == 0.851 / 8.0
    assert np.all(rho0 == 1.0) and np.all(p0 == 1e-6)


def test_batch_instances_ranges():
    inst = inputs.batch_instances(512)
    assert len(inst) == 512
    ns = np.array([(m.nx, m.ny, m.nz) for m, _ in inst])
    assert ns.min() >= 16 and ns.max() <= 96
    assert len(np.unique(ns)) > 60
    g = np.array([p.gamma for _, p in inst])
    assert g.min() >= 1.2 and g.max() <= 1.67
    kinds = [p.kind for _, p in inst]
    assert kinds[0] == inputs.PROB_SOD_X and kinds[1] == inputs.PROB_SEDOV
    pr = np.array([p.p_l if p.kind == inputs.PROB_SOD_X else p.p_blast for _, p in inst])
    assert pr.min() >= 10.0 and pr.max() <= 1e4
    assert inputs.batch_instances(4)[3][0] == inst[3][0]


def test_problem_materials_follow_the_sod_split():
    # material 1 is exactly the right state of the shock tube (logical cell
    # centres at or past x_split); one material: all zeros
    import dataclasses
    md, pd = inputs.sod_x(10, 2, 3)
    none = inputs.problem_materials(md, pd)
    assert none.dtype == np.int32 and not np.any(none)
    pm = dataclasses.replace(pd, nmat=2)
    mat = inputs.problem_materials(md, pm)
    rho0, _, _, _ = inputs.problem_prim(md, pd)
    assert np.array_equal(mat == 1, rho0 == pd.rho_r)
    assert mat.reshape(3, 2, 10)[0, 0].tolist() == [0] * 5 + [1] * 5
    # a split between two cell centres, and one past the box
    assert inputs.problem_materials(md, dataclasses.replace(pm, x_split=0.31)).reshape(3, 2, 10)[0, 0].tolist() == \
        [0] * 3 + [1] * 7
    assert not np.any(inputs.problem_materials(md, dataclasses.replace(pm, x_split=2.0)))
