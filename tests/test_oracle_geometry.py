"""Pins for the oracle's hex geometry (volume, gradient, areas, swept volumes).

Each pin is independent of the oracle's own formula: Gauss quadrature of the
trilinear Jacobian, affine invariance, Euler's theorem for homogeneous
functions, finite differences, and additivity of swept volumes.
"""
import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs

CUBE = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)


def random_hex(rng, amp=0.2):
    return CUBE + rng.uniform(-amp, amp, size=(8, 3))


def gauss_volume(X, npts=3):
    """Integral of det(dx/dxi) over the unit cube for the trilinear map with
    nodes X (local node a at xi = (a&1, a>>1&1, a>>2&1)); Gauss-Legendre
    with npts^3 points is exact for this polynomial of degree <= 2 per axis."""
    g, w = np.polynomial.legendre.leggauss(npts)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    vol = 0.0
    for r, wr in zip(g, w):
        for s, ws in zip(g, w):
            for t, wt in zip(g, w):
                J = np.zeros((3, 3))
                for a in range(8):
                    b = CUBE[a]
                    fr = (r if b[0] else 1 - r)
                    fs = (s if b[1] else 1 - s)
                    ft = (t if b[2] else 1 - t)
                    dN = np.array([(1 if b[0] else -1) * fs * ft,
                                   fr * (1 if b[1] else -1) * ft,
                                   fr * fs * (1 if b[2] else -1)])
                    J += np.outer(X[a], dN)
                vol += wr * ws * wt * np.linalg.det(J)
    return vol


def test_unit_cube():
    assert oracle.hex_volume(CUBE) == 1.0
    G = oracle.hex_volume_grad(CUBE)
    expect = np.where(CUBE > 0, 0.25, -0.25)
    assert np.array_equal(G, expect)
    assert oracle.hex_char_length(CUBE) == 1.0


def test_volume_equals_trilinear_quadrature():
    rng = np.random.default_rng(1)
    for _ in range(50):
        X = random_hex(rng, 0.3) * rng.uniform(0.1, 3.0) + rng.uniform(-5, 5, 3)
        v = oracle.hex_volume(X)
        vg = gauss_volume(X)
        assert abs(v - vg) <= 1e-12 * abs(vg)


def test_volume_affine_invariance():
    rng = np.random.default_rng(2)
    for _ in range(20):
        X = random_hex(rng)
        A = np.eye(3) + rng.uniform(-0.3, 0.3, (3, 3))
        b = rng.uniform(-2, 2, 3)
        Y = X @ A.T + b
        assert abs(oracle.hex_volume(Y) - np.linalg.det(A) * oracle.hex_volume(X)) \
            <= 1e-13 * abs(oracle.hex_volume(Y))


def test_gradient_identities_and_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(20):
        X = random_hex(rng, 0.25) + rng.uniform(-1, 1, 3)
        G = oracle.hex_volume_grad(X)
        V = oracle.hex_volume(X)
        # translation invariance: gradients sum to zero
        assert np.max(np.abs(G.sum(axis=0))) <= 1e-14
        # V is homogeneous of degree 3 in the coordinates (about any point)
        Xc = X - X.mean(axis=0)
        assert abs(np.sum(Xc * G) - 3.0 * V) <= 1e-13
        h = 1e-6
        for a in range(8):
            for d in range(3):
                Xp = X.copy(); Xp[a, d] += h
                Xm = X.copy(); Xm[a, d] -= h
                fd = (oracle.hex_volume(Xp) - oracle.hex_volume(Xm)) / (2 * h)
                assert abs(fd - G[a, d]) <= 1e-8


def test_face_areas_and_length_on_box():
    dims = np.array([0.3, 0.7, 1.9])
    X = CUBE * dims + np.array([4.0, -2.0, 1.0])
    A = oracle.hex_face_areas(X)
    areas = [dims[1] * dims[2], dims[0] * dims[2], dims[0] * dims[1]]
    for f in range(6):
        ax = f // 2
        sign = -1.0 if f % 2 == 0 else 1.0
        expect = np.zeros(3); expect[ax] = sign * areas[ax]
        assert np.allclose(A[f], expect, rtol=1e-14, atol=1e-15)
    assert abs(oracle.hex_char_length(X) - dims.min()) <= 1e-14
    # outward areas of a closed surface sum to zero on any hex
    rng = np.random.default_rng(4)
    Y = random_hex(rng, 0.3)
    assert np.max(np.abs(oracle.hex_face_areas(Y).sum(axis=0))) <= 1e-15


def _displaced_state(md, amp, seed):
    """Oracle state whose current mesh is the reference mesh moved by random
    displacements (tangential on walls)."""
    pd = inputs.ProblemDesc()
    o = oracle.Oracle.from_problem(md, pd)
    rng = np.random.default_rng(seed)
    nx, ny, nz = md.nx, md.ny, md.nz
    xr, yr, zr = o.field("xr"), o.field("yr"), o.field("zr")
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    idx = (ii.ravel(), jj.ravel(), kk.ravel())
    n = (nx, ny, nz)
    h = [(md.hi[d] - md.lo[d]) / n[d] for d in range(3)]
    cur = []
    for d, base in enumerate((xr, yr, zr)):
        disp = rng.uniform(-amp, amp, base.shape) * h[d]
        wall = (idx[d] == 0) | (idx[d] == n[d])
        cur.append(np.where(wall, base, base + disp))
    zeros = np.zeros_like(xr)
    o.set_state(cur[0], cur[1], cur[2], zeros, zeros, zeros, o.field("mn"), o.field("m"), o.field("e"))
    return o


def test_swept_volume_closure():
    """V(reference) = V(current) + sum of signed face swept volumes, per cell."""
    md = inputs.MeshDesc(4, 3, 5, lo=(0.0, -1.0, 2.0), hi=(1.0, 0.5, 3.0), jitter=0.15, seed=7)
    o = _displaced_state(md, 0.2, 11)
    dvx, dvy, dvz = o.swept_volumes()
    nx, ny, nz = md.nx, md.ny, md.nz
    xr, yr, zr = o.field("xr"), o.field("yr"), o.field("zr")
    x, y, z = o.field("x"), o.field("y"), o.field("z")

    def hexes(px, py, pz):
        P = np.stack([px, py, pz], -1).reshape(nz + 1, ny + 1, nx + 1, 3)
        out = np.zeros((nz, ny, nx))
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    X = np.array([P[k + (a >> 2 & 1), j + (a >> 1 & 1), i + (a & 1)] for a in range(8)])
                    out[k, j, i] = oracle.hex_volume(X)
        return out

    VL, VE = hexes(x, y, z), hexes(xr, yr, zr)
    net = (dvx[:, :, 1:] - dvx[:, :, :-1]) + (dvy[:, 1:, :] - dvy[:, :-1, :]) + \
          (dvz[1:, :, :] - dvz[:-1, :, :])
    assert np.max(np.abs(VE - (VL + net))) <= 1e-14 * VE.max()
    # the swept volumes are not trivially zero
    assert np.max(np.abs(dvx)) > 1e-3 * VE.mean()


def test_swept_volume_sign():
    """A face displaced towards +x in the current mesh (reference on its
    -x side) sweeps a region of the low cell: negative volume."""
    md = inputs.MeshDesc(2, 1, 1)
    o = _displaced_state(md, 0.0, 0)
    x = o.field("x")
    x[1::3] += 0.1  # the i = 1 node plane moves towards +x
    zeros = np.zeros_like(x)
    o.set_state(x, o.field("y"), o.field("z"), zeros, zeros, zeros, o.field("mn"), o.field("m"), o.field("e"))
    dvx, _, _ = o.swept_volumes()
    assert abs(dvx[0, 0, 1] - (-0.1 * 1.0 * 1.0)) <= 1e-15
