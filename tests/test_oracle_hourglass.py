"""Pins of the oracle's viscous hourglass control (c_hg > 0).

What fixes each expected value:
  * The hourglass shape vectors vanish on every linear field (the mean
    shape-function gradients reproduce linear fields), so an affine
    velocity field feels no hourglass force: one step with c_hg > 0 equals
    one step without it, to roundoff, on a jittered mesh.
  * A checkerboard velocity u_x = eps (-1)^(j+k) changes no cell volume
    (zero-energy hourglass mode of the hex): without control its kinetic
    energy persists, with control it is dissipated into internal energy.
  * Total energy: the hourglass forces enter the corner forces of both the
    velocity and the compatible energy update, so it stays exact.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2209_01983_gb300 import inputs


def state(md, pd, u, v, w):
    o = oracle.Oracle.from_problem(md, pd)
    x, y, z = inputs.mesh_nodes(md)
    o.check(o.set_state(x, y, z, u, v, w, o.field("mn"), o.field("m"), o.field("e")))
    return o


@pytest.mark.parametrize("time_order", [1, 2])
def test_affine_velocity_feels_no_hourglass_force(time_order):
    md, pd = inputs.uniform_box(7, jitter=0.15, seed=9)
    x, y, z = inputs.mesh_nodes(md)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3)) * 0.01
    u = A[0, 0] * x + A[0, 1] * y + A[0, 2] * z
    v = A[1, 0] * x + A[1, 1] * y + A[1, 2] * z
    w = A[2, 0] * x + A[2, 1] * y + A[2, 2] * z
    base = dataclasses.replace(pd, time_order=time_order)
    a = state(md, base, u, v, w)
    b = state(md, dataclasses.replace(base, c_hg=0.5), u, v, w)
    a.check(a.lagrange_step(1e-3))
    b.check(b.lagrange_step(1e-3))
    scale = max(float(np.max(np.abs(a.field(f)))) for f in "uvw")
    for f in "uvw":
        assert float(np.max(np.abs(a.field(f) - b.field(f)))) <= 1e-12 * scale, f
    assert float(np.max(np.abs(a.field("e") - b.field("e")))) <= 1e-13 * float(np.max(a.field("e")))


def checkerboard_ke(c_hg, steps=40, n=6, eps=1e-2):
    md, pd = inputs.uniform_box(n)
    pd = dataclasses.replace(pd, c_hg=c_hg, c_q=0.0, c_l=0.0)
    x, y, z = inputs.mesh_nodes(md)
    i = np.rint(x * n).astype(int)
    j = np.rint(y * n).astype(int)
    k = np.rint(z * n).astype(int)
    u = eps * (-1.0) ** (j + k) * ((i > 0) & (i < n))  # zero on the x walls
    zero = np.zeros_like(u)
    o = state(md, pd, u, zero, zero)
    d0 = o.diagnostics()
    for _ in range(steps):
        o.check(o.lagrange_step(2e-3))
    d = o.diagnostics()
    return d0, d


def test_checkerboard_mode_is_damped():
    d0, d_off = checkerboard_ke(0.0)
    _, d_on = checkerboard_ke(0.1)
    assert d_off["ke"] >= 0.9 * d0["ke"]          # a zero-energy mode: nothing resists it
    assert d_on["ke"] <= 0.5 * d_off["ke"]        # the hourglass viscosity dissipates it
    for d in (d_off, d_on):
        assert abs(d["etot"] - d0["etot"]) <= 1e-13 * d0["etot"]


def test_energy_exact_with_hourglass_control():
    md, pd = inputs.sedov_octant(10, jitter=0.15)
    for time_order in (1, 2):
        o = oracle.Oracle.from_problem(md, dataclasses.replace(pd, c_hg=0.05, time_order=time_order))
        d0 = o.diagnostics()
        rc, n = o.run(max_cycles=40, remap_every=1)
        assert rc == 0 and n == 40
        d = o.diagnostics()
        assert abs(d["etot"] - d0["etot"]) <= 1e-13 * d0["etot"]
