"""Algorithmic cost of each kernel of the cycle, per unit (cell or node).

bytes: compulsory HBM traffic of the kernel's data flow, every array it
reads or writes counted once (N_nodes ~ N_cells, so node arrays count per
cell too), in the storage precision.
flops: floating-point operations of the formulas the kernel evaluates, each
distinct quantity counted once per kernel (a multiply-add is 2, a divide or
square root 1); recomputation inside the kernel (e.g. the node gather
re-deriving corner gradients of its eight cells) is not counted.

Formula counts used below (FP64 path):
  hex volume            202  (6 faces x (9 adds node sum + 6 diagonal subs
                              + 9 cross + 5 dot + 1 accumulate) + 21 shift + 1)
  hex volume gradient   600  (24 face-corner terms x (9 weighted sum + 3 sub
                              + 9 cross + 3 accumulate) + 24 scale)
  face areas + L        122  (6 x (6 subs + 9 cross + 5 |A|^2) + max + sqrt + div)
"""

VOL, GRAD, LEN = 202, 600, 122

# General FP64 kernels (Lagrangian cycles, remap every k > 1 cycles).  The
# EoS pass evaluates the geometry once per cycle, face by face (HALF_GEOM64
# below: the corner sums, the face areas and the volume by Euler's
# relation), and keeps the 24 corner gradients (Gn) for the next step's node
# and cell passes, which read them instead of rebuilding them.
# kernel: (unit, bytes per unit FP64, flops per unit)
FP64 = {
    # x, u, mn, sigma, Gn (24 per cell) read; u, ubar, x+ written; the force
    # gathered from 8 corners (8 x 3 multiply-adds)
    "lagrange_nodes": ("node", 8 * (3 + 3 + 1 + 1 + 24 + 3 + 3 + 3), 48 + 20),
    # Gn, ubar, x+, m, e, sigma read; e, vol, rho written; work from Gn, the
    # volume at x+ for the remap's donor density
    "lagrange_cells": ("cell", 8 * (24 + 3 + 3 + 3 + 3), 48 + 5 + VOL + 1),
    # x, x_ref, rho, e read; 3 mass + 3 energy fluxes written
    "remap_faces": ("cell", 8 * (3 + 3 + 2 + 6), 3 * VOL + 6),
    # 3 mass fluxes, u, mn, x_ref read; u', mn', dKE, x written
    "remap_nodes": ("node", 8 * (3 + 3 + 1 + 3 + 3 + 1 + 1 + 3), 125),
    # 6 fluxes, m, e, dKE read; m, e written
    "remap_cells": ("cell", 8 * (6 + 2 + 1 + 2), 35),
    # x, u, m, e read; vol, rho, p, q, cs, sigma, Gn written; the geometry
    # face by face, dV/dt (48), EoS, viscosity and the CFL rate (~30)
    "eos_dt": ("cell", 8 * (3 + 3 + 2 + 6 + 24), 21 + 6 * (12 + 14 + 30 + 9) - 3 * 6 + 4 * 12 + 7 * 5 + 7 + 24
               + 48 + 30),
}

# FP64 Eulerian cycle (remap every cycle), cached reference geometry:
# corner gradients G (24 doubles per cell), V_E, L_E, 1/V_E, 1/(cfl L_E)^2
# and the reference-face terms read instead of recomputed; the side quads of
# the swept hexes computed once per mesh edge (k_ale_edges) instead of once
# per cell that uses them.
QUAD = 29  # fan term of one quad: 4-point sum 9, diagonals 6, cross 9, dot 5
# 3 side quads, Lagrangian offsets, L, origin shifts; the reference offsets
# to the neighbours are cached (read, not subtracted)
EDGES = 3 * QUAD + 9 + 3 + 6 * 7

FP64_ALE = {
    # sigma, G (24/cell), u, mn read; u, ubar, 0.5|u|^2 written
    "ale_nodes": ("node", 8 * (1 + 24 + 3 + 1 + 3 + 3 + 1), 48 + 20 + 5),
    # reference offsets to 6 neighbours (18), ubar, 3 reference-face terms
    # read; 9 side-quad terms and 3 Lagrangian + reference low-face terms
    # written
    "ale_edges": ("node", 8 * (18 + 3 + 3 + 12), EDGES + 3 * QUAD + 27 + 3),
    # G, ubar, m, e, sigma, 12 swept-hex terms read; e, 3 swept volumes written
    "ale_cells": ("cell", 8 * (24 + 3 + 3 + 12 + 1 + 3), 48 + 5 + 12 + 3),
    # 3 swept volumes, V_E, m read; V_L, rho_L written
    "ale_density": ("cell", 8 * (3 + 2 + 2), 8),
    # 3 swept volumes, rho_L, e read; 3 mass + 3 energy fluxes + 3 dual-flux parts written
    "ale_fluxes": ("cell", 8 * (3 + 2 + 6 + 3), 15),
    # 3 dual-flux parts (per cell), u, mn, 0.5|u|^2 read; u', mn', 1/mn', dKE
    # written (the node pass multiplies by 1/mn)
    "ale_remap_nodes": ("node", 8 * (3 + 3 + 1 + 1 + 3 + 1 + 1 + 1), 6 * 12 + 20),
    # 6 fluxes, m, e, dKE, u', G, V_E, L_E, 1/V_E, 1/(cfl L_E)^2 read;
    # m, 1/m, e, vol, rho, p, q, sigma written (cs is a function of e, not
    # stored; the cell pass multiplies by 1/m)
    "ale_remap_eos": ("cell", 8 * (6 + 2 + 1 + 3 + 24 + 4 + 8), 35 + 48 + 30),
}


# FP32-mixed Eulerian cycle: 4-byte fields, reference geometry recomputed
# from the structured mesh + FP32 jitter offsets (one 16-byte float4 per
# node), V_E and L_E stored; cell mass and energy are float-float (hi and lo
# arrays).  Flops are FP32.
GRAD32 = GRAD + 42      # gradient + relative coordinates of the 8 nodes
FORCE32 = 12 * 27 + 108 + 20  # 12 face terms + 18 relative node positions + update
SWEPT32 = 6 * 30 + 3 * 12 + 3 * 60 + 24  # expanded side/pair terms + displacements
MIXED_ALE = {
    # offsets (float4), sigma, u, mn read; u, ubar written
    "mix_nodes": ("node", 4 * (4 + 1 + 3 + 1 + 3 + 3), FORCE32),
    # offsets (float4), ubar, sigma, m, e (hi, lo) read; e (hi, lo), 3 swept volumes written
    "mix_cells": ("cell", 4 * (4 + 3 + 1 + 1 + 2 + 2 + 3), GRAD32 + 40 + 6 + SWEPT32),
    # swept volumes, V_E, m, e read; 3 mass + 3 energy fluxes written
    "mix_fluxes": ("cell", 4 * (3 + 3 + 6), 30),
    # 3 mass fluxes, u, mn (hi, lo) read; u', mn' (hi, lo), dKE written
    "mix_remap_nodes": ("node", 4 * (3 + 3 + 2 + 3 + 2 + 1), 125 + 6 * 9),
    # 6 fluxes, m, e (hi, lo), dKE, u', offsets (float4), V_E, L_E read;
    # m, e (hi, lo), rho, sigma written
    "mix_remap_eos": ("cell", 4 * (6 + 4 + 1 + 3 + 4 + 2 + 6), 40 + GRAD32 + 40 + 30),
}


# Jittered meshes: the reference corner gradients (24 floats per cell) are
# cached, so the cell pass and the remap+EoS pass read them instead of
# evaluating the gradient (and the remap+EoS pass no longer needs the
# offsets).
MIXED_ALE_JIT = dict(MIXED_ALE)
MIXED_ALE_JIT["mix_cells"] = ("cell", 4 * (4 + 24 + 3 + 1 + 1 + 2 + 2 + 3), 48 + 40 + 6 + SWEPT32)
MIXED_ALE_JIT["mix_remap_eos"] = ("cell", 4 * (6 + 4 + 1 + 3 + 24 + 2 + 6), 40 + 48 + 40 + 30)
# the node force gathers sum_c (sigma_c - sigma_ref) G_c(a) from the cache:
# sigma (per cell), the corner gradients (24 per cell), u, mn read; u, ubar written
MIXED_ALE_JIT["mix_nodes"] = ("node", 4 * (1 + 24 + 3 + 1 + 3 + 3), 8 * 7 + 20)


# Second-order cell remap (van Leer piecewise-linear donor cell).
SLOPE = 7  # two one-sided differences, sign test, harmonic mean
SLAB = 6   # 1 - min(nu, 1), scaled slope, add
FP64_ALE_O2 = dict(FP64_ALE)
# rho_L, e read (the neighbours' from cache); 6 slopes written
FP64_ALE_O2["ale_slopes"] = ("cell", 8 * (2 + 6), 6 * SLOPE)
# 3 swept volumes, rho_L, e, 1/V_L, 6 slopes read; 9 fluxes / dual-flux parts written
FP64_ALE_O2["ale_fluxes"] = ("cell", 8 * (3 + 3 + 6 + 9), 15 + 6 * (2 * SLAB + 1))
# 3 swept volumes, V_E, m read; V_L, rho_L, 1/V_L written
FP64_ALE_O2["ale_density"] = ("cell", 8 * (3 + 2 + 3), 9)
MIXED_O2 = {
    # 3 swept volumes, V_E, m read; V_L, rho_L written
    "mix_density": ("cell", 4 * (3 + 2 + 2), 8),
    # 3 swept volumes, rho_L, e, V_L read; 6 fluxes written (slopes in registers)
    "mix_fluxes": ("cell", 4 * (3 + 3 + 6), 3 * (2 * SLOPE + 2 * SLAB + 3)),
}


# Predictor-corrector half step (time_order 2): e^{n+1/2} from the cached
# gradient, then volume, full gradient, face areas, EoS and viscosity at
# x^{n+1/2}; the 24 corner gradients there are written for the corrector,
# whose node and cell passes read them instead of the reference ones.
# The FP64 kernel evaluates the half-step geometry face by face: per face
# the diagonals and their partner sums (12, 6 fewer on the three faces
# through node 0), the face vector and |A|^2 (14), two corner terms
# (2 x 15) and the other two from 2A (6 + 3); the corner sums accumulate
# over the last four faces (4 x 12); the volume is sum_a x_a . R_a / 72
# (Euler's relation for the cubic V: 7 dots, 6 adds, 1 scale), the 24
# gradients are scaled by 1/24.
HALF_GEOM64 = 6 * (12 + 14 + 30 + 9) - 3 * 6 + 4 * 12 + 7 * 5 + 6 + 1 + 24
FP64_PC = {
    # G, u, m, e, sigma, x_ref read; sigma, 24 half-step gradients written;
    # work 48, e 5, positions 24 + 21 (relative to node 0), geometry,
    # dV/dt 48, EoS and viscosity 40
    "ale_predict": ("cell", 8 * (24 + 3 + 3 + 3 + 3 + 24 + 1), 48 + 5 + 24 + 21 + HALF_GEOM64 + 48 + 40),
}
MIXED_PC = {
    # offsets or cached gradient, u, m, e, sigma read; sigma, 24 gradients written
    "mix_predict": ("cell", 4 * (24 + 4 + 3 + 3 + 24 + 1), 48 + 5 + 24 + VOL + GRAD + LEN + 40),
    # the node force from the half-step gradients, as on jittered meshes
    "mix_nodes": ("node", 4 * (1 + 24 + 3 + 1 + 3 + 3), 8 * 7 + 20),
}


# Viscous hourglass control: per cell the 4 patterns' sums over the 8
# nodes (positions, velocities), the velocity-gradient sums M, the rates q,
# W, and 24 corner forces written; the node and cell passes read them.
HG = 2 * 4 * 8 * 3 + 8 * 9 * 2 + 4 * (9 * 2 + 9 * 2) + 8 * (12 + 18 + 3) + 12
# FP64 Eulerian path: the projected shape vectors gamma_alpha(a) V^(1/3) of
# the reference mesh are cached (32 per cell), so per cycle the rates
# q_alpha = sum_a gamma_alpha(a) u_a (4 x 8 x 3 multiply-adds), their
# scaling by -kappa (12 + 7 for kappa and cs) and the corner forces
# f_a = sum_alpha gamma_alpha(a) q_alpha (8 x 4 x 3 multiply-adds)
HG64 = 4 * 8 * 3 * 2 + 12 + 7 + 8 * 4 * 3 * 2
FP64_HG = {
    # u, 32 cached shape vectors, rho, e read; 24 corner forces written
    "ale_hourglass": ("cell", 8 * (3 + 32 + 2 + 24), HG64),
}
MIXED_HG = {
    # offsets or cached gradient, u, V_E, rho, e read; 24 corner forces written
    "mix_hourglass": ("cell", 4 * (24 + 4 + 3 + 3 + 24), HG),
}


# Material strength (FP64): the deviatoric stress S (6) and plastic strain
# per cell.  Node pass: S of the 8 cells, S dV/dx per corner (9
# multiply-adds).  Cell pass: S, eps_p read and the new values written, the
# deviatoric work (8 x (15 + 5)), the velocity gradient (8 x 9
# multiply-adds), Steinberg-Guinan G and Y (~20), the Wilkins update (strain
# rate and spin 18, trial stress 9 x 16, J 18, return 13).  Remap: S, eps_p
# read (own and donors') and written, transported with the six face fluxes;
# the CFL speed adds G of the new state.  The general kernels also copy S,
# eps_p in the face pass for the cell remap.
_STR_CELL = 8 * 20 + 8 * 18 + 20 + 18 + 9 * 16 + 18 + 13
_STR_REMAP = 7 * (2 + 6 * 2) + 7
FP64_STRENGTH_EXTRA = {
    "lagrange_nodes": (8 * 6, 8 * 18),
    "lagrange_cells": (8 * 14, _STR_CELL),
    "eos_dt": (8 * 1, 25),
    "remap_faces": (8 * 14, 0),
    "remap_cells": (8 * 14, _STR_REMAP),
    "ale_nodes": (8 * 6, 8 * 18),
    "ale_cells": (8 * 14, _STR_CELL),
    "ale_remap_eos": (8 * 14, _STR_REMAP + 25),
}


# Several materials (FP64 general kernels), per material k: the EoS pass
# reads alpha_k, m_k, e_k and forms rho_k (2), p_k (5), c_k^2 (6) and the
# two sums (4); the cell pass reads them and q, forms rho_k, p_k and the
# work share (13) and writes e_k; the face pass reads them and V_L and
# writes the volume, mass and energy flux through each low face (6 per
# face); the cell remap reads the 9 fluxes per material of its own low
# faces (the high faces' are the neighbours' low faces), alpha_k, m_k, e_k,
# V_L, dKE, sums them (3 x 6), applies the cutoff and the kinetic-energy
# share (~18) and writes alpha_k, m_k, e_k and m, e, 1/m.
# The Eulerian kernels take the same steps: the cell pass the work split,
# the flux pass the material fluxes, the remap + EoS pass the material
# remap (9 fluxes per material instead of the 6 totals, V_L read, the
# sound speed stored) and the mixture EoS.
def materials_table(base: dict, nmat: int, path: str = "general") -> dict:
    t = dict(base)
    if path == "ale":
        extra = {"ale_cells": (8 * (4 * nmat + 1), 15 * nmat + 1),
                 # predictor-corrector: the materials' half step, their shares written
                 "ale_predict": (8 * 4 * nmat, 20 * nmat),
                 "ale_density": (8, 1),  # 1 / V_L written for the flux pass
                 "ale_fluxes": (8 * (12 * nmat + 1), 18 * nmat),
                 "ale_remap_eos": (8 * (15 * nmat - 6 + 2), 53 * nmat - 21)}
    else:
        extra = {"eos_dt": (8 * 3 * nmat, 17 * nmat + 1),
                 "lagrange_cells": (8 * (4 * nmat + 1), 15 * nmat + 1),
                 "remap_faces": (8 * (3 * nmat + 1 + 9 * nmat), 18 * nmat)}
    for k, (db, df) in extra.items():
        if k not in t:  # an option's kernel the run does not launch
            continue
        u, b, f = t[k]
        t[k] = (u, b + db, f + df)
    if path != "ale":
        t["remap_cells"] = ("cell", 8 * (9 * nmat + 3 * nmat + 2 + 3 * nmat + 3), 36 * nmat + 13)
    return t


def table(precision: str, path: str = "ale", jitter: bool = True, order: int = 1, time_order: int = 1,
          hourglass: bool = False, strength: bool = False, nmat: int = 0):
    if precision == "fp64":
        if nmat >= 2:  # the same kernels with materials (and hourglass control when asked)
            return materials_table(table(precision, path, jitter, order, time_order, hourglass), nmat, path)
        if strength:  # the same kernels with the stress module
            base = table(precision, path, jitter, order, time_order, hourglass)
            return {k: (u, b + FP64_STRENGTH_EXTRA.get(k, (0, 0))[0], f + FP64_STRENGTH_EXTRA.get(k, (0, 0))[1])
                    for k, (u, b, f) in base.items()}
        if path != "ale":
            return FP64
        t = dict(FP64_ALE_O2 if order == 2 else FP64_ALE)
        if time_order == 2:
            t.update(FP64_PC)
        if hourglass:
            t.update(FP64_HG)
        return t
    if precision == "fp32_mixed":
        t = dict(MIXED_ALE_JIT if jitter else MIXED_ALE)
        if order == 2:
            t.update(MIXED_O2)
        if time_order == 2:
            t.update(MIXED_PC)
        if hourglass:
            t.update(MIXED_HG)
        return t
    raise KeyError(precision)


def cycle_cost(precision: str, path: str = "ale", jitter: bool = True, order: int = 1, time_order: int = 1,
               hourglass: bool = False, strength: bool = False, nmat: int = 0):
    """(bytes, flops) of one full cycle per cell."""
    t = table(precision, path, jitter, order, time_order, hourglass, strength, nmat)
    return sum(v[1] for v in t.values()), sum(v[2] for v in t.values())
