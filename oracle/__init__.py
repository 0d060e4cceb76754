"""CPU oracle for the SALE hydro cycle: Python access to sale_oracle.c.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it never calls the CUDA
library: the two share only the seeded inputs of
``paper_2209_01983_gb300.inputs``.

The C source is compiled with ``-O2 -ffp-contract=off`` (no FMA contraction,
the same rounding on x86 and Arm hosts) into ``oracle/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sale_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ENEGVOL, EDT, ENAN = 0, -1, -2, -4, -5, -6

_dp = C.POINTER(C.c_double)


class Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("cfl", C.c_double), ("c_q", C.c_double),
        ("c_l", C.c_double), ("dt_growth", C.c_double), ("dt_init", C.c_double),
        ("ke_fix", C.c_int), ("reflect", C.c_int * 6), ("remap_order", C.c_int), ("time_order", C.c_int),
        ("c_hg", C.c_double),
        ("shear0", C.c_double), ("shear_dp", C.c_double), ("shear_dt", C.c_double), ("cv", C.c_double),
        ("e_ref", C.c_double), ("rho_ref", C.c_double), ("yield0", C.c_double), ("yield_max", C.c_double),
        ("hard_beta", C.c_double), ("hard_n", C.c_double),
        ("nmat", C.c_int), ("mat_gamma", C.c_double * 4), ("mat_pinf", C.c_double * 4),
    ]

STRENGTH_FIELDS = ("shear0", "shear_dp", "shear_dt", "cv", "e_ref", "rho_ref", "yield0", "yield_max",
                   "hard_beta", "hard_n")


class _State(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("nc", C.c_longlong), ("nn", C.c_longlong), ("prm", Params),
        ("x", _dp), ("y", _dp), ("z", _dp), ("xr", _dp), ("yr", _dp), ("zr", _dp),
        ("u", _dp), ("v", _dp), ("w", _dp), ("mn", _dp),
        ("m", _dp), ("e", _dp), ("vol", _dp), ("rho", _dp), ("p", _dp),
        ("q", _dp), ("cs", _dp), ("len", _dp),
        ("sxx", _dp), ("syy", _dp), ("szz", _dp), ("sxy", _dp), ("syz", _dp), ("szx", _dp), ("eps_p", _dp),
        ("t", C.c_double), ("dt", C.c_double), ("dt_last", C.c_double),
        ("cycle", C.c_longlong), ("status", C.c_int),
        ("alpha", _dp), ("mm", _dp), ("me", _dp),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its sources."""
    hdr = os.path.join(HERE, "sale_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.oracle_hex_volume.restype = C.c_double
        L.oracle_hex_volume.argtypes = [_dp]
        L.oracle_hex_volume_grad.argtypes = [_dp, _dp]
        L.oracle_hex_face_areas.argtypes = [_dp, _dp]
        L.oracle_hex_char_length.restype = C.c_double
        L.oracle_hex_char_length.argtypes = [_dp]
        L.oracle_create.restype = C.POINTER(_State)
        L.oracle_create.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, C.POINTER(Params)]
        L.oracle_destroy.argtypes = [C.POINTER(_State)]
        L.oracle_init_prim.argtypes = [C.POINTER(_State), _dp, _dp, C.c_longlong, C.c_double]
        L.oracle_init_materials.argtypes = [C.POINTER(_State), _dp, _dp, C.POINTER(C.c_int), C.c_longlong,
                                            C.c_double]
        L.oracle_set_materials.argtypes = [C.POINTER(_State), _dp, _dp, _dp]
        L.oracle_set_state.argtypes = [C.POINTER(_State)] + [_dp] * 9 + [C.c_double, C.c_double]
        L.oracle_eos.argtypes = [C.POINTER(_State)]
        L.oracle_cfl_dt.restype = C.c_double
        L.oracle_cfl_dt.argtypes = [C.POINTER(_State)]
        L.oracle_lagrange_step.argtypes = [C.POINTER(_State), C.c_double]
        L.oracle_remap_step.argtypes = [C.POINTER(_State)]
        L.oracle_swept_volumes.argtypes = [C.POINTER(_State), _dp, _dp, _dp]
        L.oracle_run.argtypes = [C.POINTER(_State), C.c_double, C.c_longlong, C.c_int,
                                 C.POINTER(C.c_longlong)]
        L.oracle_diagnostics.argtypes = [C.POINTER(_State), _dp]
        L.oracle_steinberg.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]
        L.oracle_stress_update.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _hexarr(X) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(8, 3))
    return X


def hex_volume(X) -> float:
    """Exact volume of the trilinear hex with local nodes X[a] (a = di+2dj+4dk)."""
    return lib().oracle_hex_volume(_ptr(_hexarr(X)))


def hex_volume_grad(X) -> np.ndarray:
    G = np.zeros((8, 3))
    lib().oracle_hex_volume_grad(_ptr(_hexarr(X)), _ptr(G))
    return G


def hex_face_areas(X) -> np.ndarray:
    A = np.zeros((6, 3))
    lib().oracle_hex_face_areas(_ptr(_hexarr(X)), _ptr(A))
    return A


def hex_char_length(X) -> float:
    return lib().oracle_hex_char_length(_ptr(_hexarr(X)))


def steinberg(params: Params, p, rho, e, eps_p):
    """(G, Y) of the Steinberg-Guinan model for one cell state."""
    G, Y = C.c_double(0.0), C.c_double(0.0)
    lib().oracle_steinberg(C.byref(params), p, rho, e, eps_p, C.byref(G), C.byref(Y))
    return G.value, Y.value


def stress_update(S6, L, dt, G, Y):
    """One Wilkins stress update: (S_new[6], plastic strain added)."""
    S6 = np.ascontiguousarray(S6, dtype=np.float64).reshape(6)
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(9)
    out = np.zeros(6)
    deps = C.c_double(0.0)
    lib().oracle_stress_update(_ptr(S6), _ptr(L), dt, G, Y, _ptr(out), C.byref(deps))
    return out, deps.value


def params_from(pd, reflect=(1, 1, 1, 1, 1, 1)) -> Params:
    p = Params()
    p.gamma, p.cfl, p.c_q, p.c_l = pd.gamma, pd.cfl, pd.c_q, pd.c_l
    p.dt_growth = pd.dt_growth
    p.dt_init = pd.dt_init if math.isfinite(pd.dt_init) else 0.0
    p.ke_fix = int(pd.ke_fix)
    for i in range(6):
        p.reflect[i] = int(reflect[i])
    p.remap_order = int(getattr(pd, "remap_order", 1))
    p.time_order = int(getattr(pd, "time_order", 1))
    p.c_hg = float(getattr(pd, "c_hg", 0.0))
    for name in STRENGTH_FIELDS:
        setattr(p, name, float(getattr(pd, name, 0.0)))
    p.nmat = int(getattr(pd, "nmat", 0))
    for k, (g, pinf) in enumerate(zip(getattr(pd, "mat_gamma", (1.4,) * 4), getattr(pd, "mat_pinf", (0.0,) * 4))):
        p.mat_gamma[k], p.mat_pinf[k] = float(g), float(pinf)
    return p


class Oracle:
    """One oracle state (owns C memory)."""

    NODE_FIELDS = ("x", "y", "z", "xr", "yr", "zr", "u", "v", "w", "mn")
    CELL_FIELDS = ("m", "e", "vol", "rho", "p", "q", "cs", "len", "sxx", "syy", "szz", "sxy", "syz", "szx", "eps_p")

    def __init__(self, nx, ny, nz, nodes, params: Params):
        x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in nodes)
        self._params = params
        self._s = lib().oracle_create(nx, ny, nz, _ptr(x), _ptr(y), _ptr(z), C.byref(params))
        if not self._s:
            raise MemoryError("oracle_create failed")
        self.nx, self.ny, self.nz = nx, ny, nz

    @classmethod
    def from_problem(cls, md, pd):
        """Build and initialise from the seeded inputs (mesh + primitives)."""
        from paper_2209_01983_gb300 import inputs
        o = cls(md.nx, md.ny, md.nz, inputs.mesh_nodes(md), params_from(pd, md.reflect))
        rho0, p0, dep_cell, dep_e = inputs.problem_prim(md, pd)
        if getattr(pd, "nmat", 0) >= 2:
            mat = np.ascontiguousarray(inputs.problem_materials(md, pd), dtype=np.int32)
            o.check(lib().oracle_init_materials(o._s, _ptr(rho0), _ptr(p0), mat.ctypes.data_as(C.POINTER(C.c_int)),
                                                dep_cell, dep_e))
        else:
            o.check(lib().oracle_init_prim(o._s, _ptr(rho0), _ptr(p0), dep_cell, dep_e))
        return o

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            lib().oracle_destroy(s)
            self._s = None

    @property
    def s(self):
        return self._s.contents

    def check(self, rc):
        if rc != OK:
            raise RuntimeError(f"oracle status {rc}")
        return rc

    def field(self, name) -> np.ndarray:
        """A node or cell field; material fields are alpha<k> (volume
        fraction), m<k> (mass) and e<k> (specific internal energy) of
        material k."""
        mat = re.fullmatch(r"(alpha|m|e)(\d)", name)
        if mat:
            k, nc = int(mat.group(2)), self.s.nc
            if not 0 <= k < max(self.s.prm.nmat, 0) or self.s.prm.nmat < 2:
                raise KeyError(name)
            ptr = getattr(self.s, {"alpha": "alpha", "m": "mm", "e": "me"}[mat.group(1)])
            return np.ctypeslib.as_array(ptr, shape=(self.s.prm.nmat * nc,))[k * nc:(k + 1) * nc].copy()
        n = self.s.nn if name in self.NODE_FIELDS else self.s.nc
        ptr = getattr(self.s, name)
        return np.ctypeslib.as_array(ptr, shape=(n,)).copy()

    def set_materials(self, alpha, m, e):
        """Per-material fields, one array per material each (see
        oracle_set_materials); returns the status."""
        arrs = [np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64) for a in f]))
                for f in (alpha, m, e)]
        return lib().oracle_set_materials(self._s, *[_ptr(a) for a in arrs])

    def set_state(self, x, y, z, u, v, w, mn, m, e, t=0.0, dt_last=math.inf):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, u, v, w, mn, m, e)]
        return lib().oracle_set_state(self._s, *[_ptr(a) for a in arrs], t, dt_last)

    def lagrange_step(self, dt):
        return lib().oracle_lagrange_step(self._s, dt)

    def remap_step(self):
        return lib().oracle_remap_step(self._s)

    def eos(self):
        return lib().oracle_eos(self._s)

    def cfl_dt(self):
        return lib().oracle_cfl_dt(self._s)

    def run(self, t_end=math.inf, max_cycles=1 << 60, remap_every=0):
        done = C.c_longlong(0)
        rc = lib().oracle_run(self._s, t_end, max_cycles, remap_every, C.byref(done))
        return rc, done.value

    def swept_volumes(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        dvx = np.zeros((nz, ny, nx + 1))
        dvy = np.zeros((nz, ny + 1, nx))
        dvz = np.zeros((nz + 1, ny, nx))
        lib().oracle_swept_volumes(self._s, _ptr(dvx), _ptr(dvy), _ptr(dvz))
        return dvx, dvy, dvz

    def diagnostics(self) -> dict:
        out = np.zeros(7)
        lib().oracle_diagnostics(self._s, _ptr(out))
        keys = ("mass", "mom_x", "mom_y", "mom_z", "ie", "ke", "etot")
        d = dict(zip(keys, out.tolist()))
        d.update(t=self.s.t, dt=self.s.dt, cycle=self.s.cycle, status=self.s.status)
        return d
