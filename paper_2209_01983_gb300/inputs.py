"""Seeded synthetic inputs for the SALE hydro cycle (no method arithmetic).

This module is the one piece shared by the CUDA library's callers and the
CPU oracle.  It produces only *inputs*: node coordinates of the structured
hex mesh and per-cell primitive initial states (density, pressure, an
optional energy deposit).  Everything derived from them -- volumes, masses,
specific energies, node masses -- is computed independently on each side.

Problems follow the ones the paper names: the Sod shock tube and the
Sedov-Taylor blast (ScalSALE, arXiv 2209.01983, Sec. I-D and Sec. IV).

Random numbers use SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) as a counter-based generator:
draw k of stream `seed` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15).  The C
library implements the same definition for its own mesh jitter.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Problem kinds (same values as the C ABI's SALE_PROB_*).
PROB_SOD_X = 0
PROB_SEDOV = 1
PROB_UNIFORM = 2


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: output number k (uint64 array) of stream seed."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, k: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class MeshDesc:
    """Structured hex mesh on the box [lo, hi] with nx*ny*nz cells.

    jitter: each node coordinate gets an independent offset uniform in
    +-jitter*h along that axis (none normal to a boundary plane it lies on).
    reflect: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi walls (1 = reflecting).
    """
    nx: int
    ny: int
    nz: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    jitter: float = 0.0
    seed: int = 2209
    reflect: tuple = (1, 1, 1, 1, 1, 1)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nnode(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)


@dataclass
class ProblemDesc:
    """Initial state and scheme parameters (same fields as sale_problem_desc)."""
    kind: int = PROB_UNIFORM
    gamma: float = 1.4
    rho_l: float = 1.0
    p_l: float = 1.0
    rho_r: float = 0.125
    p_r: float = 0.1
    x_split: float = 0.5
    rho_bg: float = 1.0
    p_bg: float = 1.0
    rho_blast: float = 1.0
    p_blast: float = 1.0
    e_deposit: float = 0.0
    cfl: float = 0.3
    c_q: float = 1.0
    c_l: float = 0.5
    dt_init: float = math.inf
    dt_growth: float = 1.1
    ke_fix: int = 1
    remap_order: int = 1  # cell remap: 1 donor cell, 2 van Leer piecewise linear
    time_order: int = 1   # Lagrange step: 1 single stage, 2 predictor-corrector
    c_hg: float = 0.0     # viscous hourglass coefficient (0: no hourglass control)
    # material strength, Steinberg-Guinan model (shear0 = 0: none)
    shear0: float = 0.0     # shear modulus G0 at the reference state
    shear_dp: float = 0.0   # dG/dp
    shear_dt: float = 0.0   # dG/dT
    cv: float = 1.0         # specific heat: T - T_ref = (e - e_ref) / cv
    e_ref: float = 0.0      # specific internal energy at the reference temperature
    rho_ref: float = 1.0    # reference density
    yield0: float = 0.0     # Y0
    yield_max: float = 0.0  # Ymax
    hard_beta: float = 0.0  # work-hardening coefficient
    hard_n: float = 0.0     # work-hardening exponent
    # materials (nmat <= 1: the single ideal gas of `gamma`); with nmat >= 2
    # material k has the stiffened-gas EoS (mat_gamma[k], mat_pinf[k])
    nmat: int = 0
    mat_gamma: tuple = (1.4, 1.4, 1.4, 1.4)
    mat_pinf: tuple = (0.0, 0.0, 0.0, 0.0)


def mesh_nodes(md: MeshDesc):
    """Node coordinates (x, y, z), each of length nnode, x index fastest.

    Uniform node i on axis d sits at lo[d] + i * h[d], h = (hi - lo) / n,
    then gets its jitter offset ((2u - 1) * jitter) * h[d], with u the
    SplitMix64 draw number 3 * node + d of stream `seed`.
    """
    n = (md.nx, md.ny, md.nz)
    h = [(md.hi[d] - md.lo[d]) / n[d] for d in range(3)]
    kk, jj, ii = np.meshgrid(np.arange(md.nz + 1), np.arange(md.ny + 1),
                             np.arange(md.nx + 1), indexing="ij")
    idx = (ii, jj, kk)
    node = np.arange(md.nnode, dtype=np.uint64).reshape(ii.shape)
    out = []
    for d in range(3):
        c = md.lo[d] + idx[d].astype(np.float64) * h[d]
        if md.jitter != 0.0:
            u = uniform01(md.seed, node * np.uint64(3) + np.uint64(d))
            off = ((2.0 * u - 1.0) * md.jitter) * h[d]
            interior = (idx[d] > 0) & (idx[d] < n[d])
            c = np.where(interior, c + off, c)
        out.append(np.ascontiguousarray(c.reshape(-1)))
    return tuple(out)


def problem_prim(md: MeshDesc, pd: ProblemDesc):
    """Per-cell primitive initial state.

    Returns (rho0, p0, deposit_cell, deposit_energy).  A deposit_cell >= 0
    means that cell's specific internal energy is set to
    deposit_energy / (its mass) by whoever builds the state.

    SOD_X: a cell is on the left state when lo_x + (i + 0.5) * h_x < x_split
    (its logical centre), else on the right state.
    SEDOV: background (rho_bg, p_bg); the origin cell (0,0,0) holds either
    the energy deposit (e_deposit > 0) or the primitive (rho_blast, p_blast).
    UNIFORM: (rho_bg, p_bg) everywhere.
    """
    nc = md.ncell
    if pd.kind == PROB_SOD_X:
        hx = (md.hi[0] - md.lo[0]) / md.nx
        i = np.arange(md.nx, dtype=np.float64)
        left_i = (md.lo[0] + (i + 0.5) * hx) < pd.x_split
        left = np.broadcast_to(left_i[None, None, :], (md.nz, md.ny, md.nx)).reshape(-1)
        rho0 = np.where(left, pd.rho_l, pd.rho_r).astype(np.float64)
        p0 = np.where(left, pd.p_l, pd.p_r).astype(np.float64)
        return rho0, p0, -1, 0.0
    rho0 = np.full(nc, pd.rho_bg, dtype=np.float64)
    p0 = np.full(nc, pd.p_bg, dtype=np.float64)
    if pd.kind == PROB_SEDOV:
        if pd.e_deposit > 0.0:
            return rho0, p0, 0, pd.e_deposit
        rho0[0] = pd.rho_blast
        p0[0] = pd.p_blast
        return rho0, p0, -1, 0.0
    if pd.kind == PROB_UNIFORM:
        return rho0, p0, -1, 0.0
    raise ValueError(f"unknown problem kind {pd.kind}")


def problem_materials(md: MeshDesc, pd: ProblemDesc) -> np.ndarray:
    """Material of every cell (int32) for nmat >= 2: material 1 where the
    logical cell centre lo_x + (i + 0.5) * h_x >= x_split (the right state
    of SOD_X), material 0 elsewhere.  All zeros for nmat <= 1."""
    if pd.nmat < 2:
        return np.zeros(md.ncell, dtype=np.int32)
    hx = (md.hi[0] - md.lo[0]) / md.nx
    i = np.arange(md.nx, dtype=np.float64)
    right_i = ~((md.lo[0] + (i + 0.5) * hx) < pd.x_split)
    right = np.broadcast_to(right_i[None, None, :], (md.nz, md.ny, md.nx)).reshape(-1)
    return right.astype(np.int32)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

# Sedov energy constant for gamma = 1.4: E = alpha * rho * R^5 / t^2 with
# alpha ~= 0.851 puts the full-space shock at R = 1 at t = 1.  The octant
# domain holds one eighth of the full-space blast energy.
SEDOV_ALPHA_G14 = 0.851


def sod_x(nx=100, ny=4, nz=4):
    """3D Sod shock tube along x on [0,1] x [0,0.04]^2, reflecting walls."""
    md = MeshDesc(nx, ny, nz, lo=(0.0, 0.0, 0.0), hi=(1.0, 0.04, 0.04))
    pd = ProblemDesc(kind=PROB_SOD_X, gamma=1.4, rho_l=1.0, p_l=1.0,
                     rho_r=0.125, p_r=0.1, x_split=0.5)
    return md, pd


def sedov_octant(n=64, jitter=0.0, seed=2209, extent=1.2):
    """Sedov blast in the octant [0, extent]^3: rho = 1, p = 1e-6, energy
    0.851 / 8 in the origin cell, symmetry planes at x = y = z = 0 and
    reflecting outer walls."""
    md = MeshDesc(n, n, n, lo=(0.0, 0.0, 0.0), hi=(extent, extent, extent),
                  jitter=jitter, seed=seed)
    pd = ProblemDesc(kind=PROB_SEDOV, gamma=1.4, rho_bg=1.0, p_bg=1e-6,
                     e_deposit=SEDOV_ALPHA_G14 / 8.0)
    return md, pd


def uniform_box(n=8, rho=1.0, p=1.0, jitter=0.0, seed=2209):
    md = MeshDesc(n, n, n, jitter=jitter, seed=seed)
    pd = ProblemDesc(kind=PROB_UNIFORM, rho_bg=rho, p_bg=p)
    return md, pd


def batch_instances(count=512, seed=2209, nmin=16, nmax=96):
    """Independent shock-tube / Sedov-like instances on [0,1]^3.

    Per instance k (draws 8k .. 8k+5 of stream `seed`): nx, ny, nz uniform
    in nmin..nmax; gamma uniform in [1.2, 1.67]; pressure ratio
    10^U[1,4]; density ratio U[1,10].  Even k: shock tube along x with the
    high state (dr, pr) on the left and (1, 1) on the right, diaphragm at
    x = 0.5.  Odd k: Sedov-like, background (1, 1) with (dr, pr) in the
    origin cell.
    """
    out = []
    span = nmax - nmin + 1
    for k in range(count):
        u = uniform01(seed, np.arange(8 * k, 8 * k + 6, dtype=np.uint64))
        nx, ny, nz = (nmin + min(int(u[d] * span), span - 1) for d in range(3))
        gamma = 1.2 + u[3] * (1.67 - 1.2)
        pr = 10.0 ** (1.0 + 3.0 * u[4])
        dr = 1.0 + 9.0 * u[5]
        md = MeshDesc(nx, ny, nz)
        if k % 2 == 0:
            pd = ProblemDesc(kind=PROB_SOD_X, gamma=gamma, rho_l=dr, p_l=pr,
                             rho_r=1.0, p_r=1.0, x_split=0.5)
        else:
            pd = ProblemDesc(kind=PROB_SEDOV, gamma=gamma, rho_bg=1.0, p_bg=1.0,
                             rho_blast=dr, p_blast=pr, e_deposit=0.0)
        out.append((md, pd))
    return out
