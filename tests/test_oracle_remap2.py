"""Pins of the oracle's second-order cell remap (van Leer's limited
piecewise-linear donor cell, averaged over the swept slab).

What fixes each expected value:
  * A linear density field translated with the mesh and remapped back: the
    cell averages of a linear field are its values at the cell centres, and
    van Leer's slope of linear data is its exact slope, so the remapped
    interior cells hold the translated field exactly: rho - beta * delta.
    The first-order donor cell smears it (checked to fail the same bar).
  * A translated step: the limited profile creates no new extrema.
  * Mass and total energy: conserved to roundoff (flux form).
  * Eulerian Sod tube against the exact Riemann solution: the second-order
    remap is closer to it than the first-order one.
"""
import dataclasses

import numpy as np
import pytest

import exact_riemann as er
import oracle
from paper_2209_01983_gb300 import inputs


def translated_box(order, rho_of_x, nx=14, delta_frac=0.3, steps=1):
    """Box nx x 3 x 3 of unit cells, uniform e, density rho_of_x(cell centre
    x); every node shifted by delta in x, then one remap back (repeated
    `steps` times, each step starting from the last remapped masses)."""
    md = inputs.MeshDesc(nx, 3, 3, lo=(0.0, 0.0, 0.0), hi=(float(nx), 3.0, 3.0))
    pd = dataclasses.replace(inputs.ProblemDesc(), remap_order=order)
    o = oracle.Oracle.from_problem(md, pd)
    xr, yr, zr = inputs.mesh_nodes(md)
    delta = delta_frac
    xc = np.arange(nx) + 0.5 + delta  # Lagrangian cell centres
    m = np.tile(rho_of_x(xc), 9)  # unit cells: mass = density
    nn = md.nnode
    z = np.zeros(nn)
    mn = np.ones(nn)
    for _ in range(steps):
        o.check(o.set_state(xr + delta, yr, zr, z, z, z, mn, m, np.full(md.ncell, 2.5)))
        o.check(o.remap_step())
        m = o.field("m")
    return m.reshape(3, 3, nx), delta, xc - delta


@pytest.mark.parametrize("beta", [0.05, -0.02])
def test_linear_profile_translated_exactly(beta):
    m, delta, xref = translated_box(2, lambda x: 1.0 + beta * x)
    want = 1.0 + beta * xref  # the linear field at the reference centres
    inner = slice(2, m.shape[2] - 1)
    assert np.max(np.abs(m[:, :, inner] - want[inner])) <= 1e-13


def test_quadratic_profile_second_order_error():
    # cell values f(c) + f''/24 are the cell averages of f(x) = a + b x^2, so
    # the exact remap gives the same at the reference centres.  First-order upwind
    # leaves delta (1 - delta) f''/2 (unit cells); the limited linear profile
    # removes almost all of it away from the extremum at x = 0.
    a, b = 0.5, 0.01
    f = lambda x: a + b * x ** 2
    for frac in (0.3, 0.55):
        avg = lambda x: f(x) + b / 12.0
        m1, delta, xref = translated_box(1, avg, delta_frac=frac)
        m2, _, _ = translated_box(2, avg, delta_frac=frac)
        inner = slice(2, m1.shape[2] - 1)
        e1 = m1[0, 0, inner] - avg(xref[inner])
        e2 = m2[0, 0, inner] - avg(xref[inner])
        assert np.allclose(e1, delta * (1 - delta) * b, rtol=1e-10, atol=1e-15)
        assert np.max(np.abs(e2)) <= 0.1 * np.max(np.abs(e1))
        assert np.max(np.abs(e2[3:])) <= 0.01 * np.max(np.abs(e1))


def test_translated_step_keeps_bounds_and_is_closer_to_exact():
    # The x-lo wall lets nothing in, so after n steps of delta the exact cell
    # averages are those of the initial step shifted by n delta with vacuum
    # behind it.  The limited profile creates no new extrema and lands
    # closer to them than the first-order donor cell.
    step = lambda x: np.where(x < 5.0, 1.0, 0.125)
    nx, n = 24, 12
    edges = np.arange(nx + 1, dtype=float)

    def exact(shift):
        def prim(x):  # integral of the shifted profile from 0 to x
            x = np.clip(x, shift, None)
            return np.minimum(x, 5.0 + shift) - shift + 0.125 * np.clip(x - 5.0 - shift, 0.0, None)
        return np.diff(prim(edges))

    for frac in (0.1, 0.3, 0.6):
        m1, _, _ = translated_box(1, step, nx=nx, delta_frac=frac, steps=n)
        m2, _, _ = translated_box(2, step, nx=nx, delta_frac=frac, steps=n)
        inner = m2[:, :, :-2]  # the last cells collect what the x-hi wall keeps in
        assert inner.min() >= 0.0 and inner.max() <= 1.0 + 1e-14
        want = exact(n * frac)[:-2]
        l1_1 = np.sum(np.abs(m1[0, 0, :-2] - want))
        l1_2 = np.sum(np.abs(m2[0, 0, :-2] - want))
        assert l1_2 < 0.9 * l1_1, (frac, l1_1, l1_2)


@pytest.mark.parametrize("jitter", [0.0, 0.15])
def test_second_order_ale_conserves(jitter):
    md, pd = inputs.sedov_octant(12, jitter=jitter)
    pd = dataclasses.replace(pd, remap_order=2)
    o = oracle.Oracle.from_problem(md, pd)
    d0 = o.diagnostics()
    rc, n = o.run(max_cycles=60, remap_every=1)
    assert rc == 0 and n == 60
    d = o.diagnostics()
    assert abs(d["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d["etot"] - d0["etot"]) <= 1e-12 * d0["etot"]
    assert np.all(o.field("rho") > 0) and np.all(o.field("e") > 0)


def eulerian_sod_l1(order, nx=100):
    md, pd = inputs.sod_x(nx, 4, 4)
    pd = dataclasses.replace(pd, remap_order=order)
    o = oracle.Oracle.from_problem(md, pd)
    rc, _ = o.run(t_end=0.2, remap_every=1)
    assert rc == 0
    rho = o.field("rho").reshape(4, 4, nx)[0, 0]
    xc = (np.arange(nx) + 0.5) / nx  # the reference mesh
    rex, _, _ = er.solution(xc, 0.2, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    return float(np.sum(np.abs(rho - rex)) / nx)


def test_second_order_remap_is_closer_to_exact_sod():
    l1_1, l1_2 = eulerian_sod_l1(1), eulerian_sod_l1(2)
    assert l1_2 < 0.8 * l1_1, (l1_1, l1_2)
