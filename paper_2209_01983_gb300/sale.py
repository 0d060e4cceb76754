"""Thin ctypes binding of libsale_gb300.so (include/sale.h), same names.

Only argument marshalling happens here: every step of the hydro cycle runs
in the library's CUDA kernels.  PyTorch supplies the device buffer and the
CUDA stream.  If the library is not built the import of this module fails
loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsale_gb300.so")

SALE_OK, SALE_EINVAL, SALE_ENOMEM, SALE_ECUDA = 0, -1, -2, -3
SALE_ENEGVOL, SALE_EDT, SALE_ENAN, SALE_ETIMEOUT, SALE_ESTATE = -4, -5, -6, -7, -8
SALE_FP64, SALE_FP32_MIXED = 0, 1

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(LIB_PATH)


class sale_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("jitter", C.c_double),
                ("seed", C.c_ulonglong), ("reflect", C.c_int * 6)]


class sale_problem_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double),
                ("rho_l", C.c_double), ("p_l", C.c_double), ("rho_r", C.c_double),
                ("p_r", C.c_double), ("x_split", C.c_double),
                ("rho_bg", C.c_double), ("p_bg", C.c_double), ("rho_blast", C.c_double),
                ("p_blast", C.c_double), ("e_deposit", C.c_double),
                ("cfl", C.c_double), ("c_q", C.c_double), ("c_l", C.c_double),
                ("dt_init", C.c_double), ("dt_growth", C.c_double), ("ke_fix", C.c_int),
                ("remap_order", C.c_int), ("time_order", C.c_int), ("c_hg", C.c_double),
                ("shear0", C.c_double), ("shear_dp", C.c_double), ("shear_dt", C.c_double), ("cv", C.c_double),
                ("e_ref", C.c_double), ("rho_ref", C.c_double), ("yield0", C.c_double), ("yield_max", C.c_double),
                ("hard_beta", C.c_double), ("hard_n", C.c_double),
                ("nmat", C.c_int), ("mat_gamma", C.c_double * 4), ("mat_pinf", C.c_double * 4)]


class sale_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("cycle", C.c_longlong),
                ("mass", C.c_double), ("mom", C.c_double * 3), ("ie", C.c_double),
                ("ke", C.c_double), ("etot", C.c_double), ("status", C.c_int)]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


sale_mesh_create = _sig("sale_mesh_create", C.c_int, [C.POINTER(sale_mesh_desc), C.POINTER(_vp)])
sale_mesh_destroy = _sig("sale_mesh_destroy", None, [_vp])
sale_mesh_nodes = _sig("sale_mesh_nodes", C.c_int, [_vp, _dp, C.c_size_t])
sale_state_bytes = _sig("sale_state_bytes", C.c_size_t, [_vp, C.c_int])
sale_state_bytes_for = _sig("sale_state_bytes_for", C.c_size_t, [_vp, _vp, C.c_int])
sale_state_init = _sig("sale_state_init", C.c_int,
                       [_vp, C.POINTER(sale_problem_desc), C.c_int, _vp, C.c_size_t, _vp, C.POINTER(_vp)])
sale_state_destroy = _sig("sale_state_destroy", None, [_vp])
sale_lagrange_step = _sig("sale_lagrange_step", C.c_int, [_vp, C.c_double])
sale_remap_step = _sig("sale_remap_step", C.c_int, [_vp])
sale_run_to_time = _sig("sale_run_to_time", C.c_int,
                        [_vp, C.c_double, C.c_longlong, C.c_int, C.POINTER(C.c_longlong)])
sale_diagnostics = _sig("sale_diagnostics", C.c_int, [_vp, C.POINTER(sale_diag)])
sale_copy_field = _sig("sale_copy_field", C.c_int, [_vp, C.c_char_p, _dp, C.c_size_t])
sale_set_field = _sig("sale_set_field", C.c_int, [_vp, C.c_char_p, _dp, C.c_size_t])
sale_refresh = _sig("sale_refresh", C.c_int, [_vp])
sale_state_dims = _sig("sale_state_dims", C.c_int, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)])
sale_profile = _sig("sale_profile", C.c_int, [_vp, C.c_int])
sale_profile_read = _sig("sale_profile_read", C.c_int,
                         [_vp, _dp, C.POINTER(C.c_longlong), C.c_int, C.c_int])
sale_kernel_count = _sig("sale_kernel_count", C.c_int, [])
sale_kernel_name = _sig("sale_kernel_name", C.c_char_p, [C.c_int])
sale_batch_bytes = _sig("sale_batch_bytes", C.c_size_t, [C.c_int, C.POINTER(sale_mesh_desc), C.c_int])
sale_batch_create = _sig("sale_batch_create", C.c_int,
                         [C.c_int, C.POINTER(sale_mesh_desc), C.POINTER(sale_problem_desc), C.c_int, _vp,
                          C.c_size_t, _vp, C.POINTER(_vp)])
sale_batch_run = _sig("sale_batch_run", C.c_int, [_vp, C.c_longlong, C.c_int, C.POINTER(C.c_longlong)])
sale_batch_state = _sig("sale_batch_state", _vp, [_vp, C.c_int])
sale_batch_destroy = _sig("sale_batch_destroy", None, [_vp])
sale_tile_shape = _sig("sale_tile_shape", C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)])
sale_set_tiling = _sig("sale_set_tiling", C.c_int, [_vp, C.c_int])
sale_batch_set_schedule = _sig("sale_batch_set_schedule", C.c_int, [_vp, C.c_int, C.c_int])
sale_remap_static = _sig("sale_remap_static", C.c_int,
                         [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, _vp, _vp, _vp, _vp,
                          _vp, _vp, _vp, _vp, _vp])
SALE_STATIC_MAX_CELLS = 65536
SALE_STATIC_MAX_NODES = 131072
sale_fma_probe = _sig("sale_fma_probe", C.c_int, [C.c_int, _vp, C.c_size_t, _vp, C.POINTER(C.c_double)])
sale_last_error = _sig("sale_last_error", C.c_char_p, [])

#: every symbol declared in include/sale.h
EXPORTS = ("sale_fma_probe", "sale_mesh_create", "sale_mesh_destroy", "sale_mesh_nodes", "sale_state_bytes", "sale_state_bytes_for",
           "sale_state_init", "sale_state_destroy", "sale_lagrange_step", "sale_remap_step",
           "sale_run_to_time", "sale_diagnostics", "sale_copy_field", "sale_set_field",
           "sale_refresh", "sale_state_dims", "sale_profile", "sale_profile_read",
           "sale_kernel_count", "sale_kernel_name", "sale_remap_static", "sale_batch_bytes",
           "sale_batch_create", "sale_batch_run", "sale_batch_state", "sale_batch_destroy",
           "sale_tile_shape", "sale_set_tiling", "sale_batch_set_schedule", "sale_last_error")


class SaleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sale status {code}: {msg}")
        self.code = code


def check(rc):
    if rc != SALE_OK:
        raise SaleError(rc, sale_last_error().decode(errors="replace"))
    return rc


def mesh_desc(md: inputs.MeshDesc) -> sale_mesh_desc:
    d = sale_mesh_desc()
    d.nx, d.ny, d.nz = md.nx, md.ny, md.nz
    for a in range(3):
        d.lo[a], d.hi[a] = md.lo[a], md.hi[a]
    d.jitter = md.jitter
    d.seed = md.seed
    for f in range(6):
        d.reflect[f] = int(md.reflect[f])
    return d


def problem_desc(pd: inputs.ProblemDesc) -> sale_problem_desc:
    p = sale_problem_desc()
    for name, _ in sale_problem_desc._fields_:
        v = getattr(pd, name)
        if name in ("mat_gamma", "mat_pinf"):
            for k in range(4):
                getattr(p, name)[k] = float(v[k])
            continue
        setattr(p, name, int(v) if name in ("kind", "ke_fix", "remap_order", "time_order", "nmat") else float(v))
    if not math.isfinite(p.dt_init):
        p.dt_init = 0.0
    return p


class Mesh:
    def __init__(self, md: inputs.MeshDesc):
        self.md = md
        self._h = _vp()
        check(sale_mesh_create(C.byref(mesh_desc(md)), C.byref(self._h)))

    def nodes(self):
        n = 3 * self.md.nnode
        out = np.empty(n)
        check(sale_mesh_nodes(self._h, out.ctypes.data_as(_dp), n))
        return out[: n // 3], out[n // 3: 2 * n // 3], out[2 * n // 3:]

    def __del__(self):
        if getattr(self, "_h", None):
            sale_mesh_destroy(self._h)
            self._h = None


class State:
    """A state on one GPU: torch owns the device buffer and the stream."""

    NODE = ("x", "y", "z", "u", "v", "w", "mn", "xref", "yref", "zref")

    def __init__(self, md: inputs.MeshDesc, pd: inputs.ProblemDesc, precision=SALE_FP64,
                 device="cuda", stream=None):
        import torch

        self.md, self.pd = md, pd
        self.mesh = Mesh(md)
        self._prob = problem_desc(pd)
        nbytes = sale_state_bytes_for(self.mesh._h, C.byref(self._prob), precision)
        if nbytes == 0:
            raise SaleError(SALE_EINVAL, f"unsupported precision {precision}")
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self._h = _vp()
        check(sale_state_init(self.mesh._h, C.byref(self._prob), precision,
                              _vp(self.buffer.data_ptr()), nbytes, _vp(self.stream.cuda_stream),
                              C.byref(self._h)))
        self.ncell, self.nnode = md.ncell, md.nnode

    def close(self):
        if getattr(self, "_h", None):
            sale_state_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def lagrange_step(self, dt=0.0):
        check(sale_lagrange_step(self._h, dt))

    def remap_step(self):
        check(sale_remap_step(self._h))

    def run_to_time(self, t_end=math.inf, max_cycles=(1 << 62), remap_every=0):
        done = C.c_longlong(0)
        check(sale_run_to_time(self._h, t_end, max_cycles, remap_every, C.byref(done)))
        return done.value

    def diagnostics(self) -> dict:
        d = sale_diag()
        check(sale_diagnostics(self._h, C.byref(d)))
        return dict(t=d.t, dt=d.dt, cycle=d.cycle, mass=d.mass, mom_x=d.mom[0], mom_y=d.mom[1],
                    mom_z=d.mom[2], ie=d.ie, ke=d.ke, etot=d.etot, status=d.status)

    def field(self, name) -> np.ndarray:
        n = self.nnode if name in self.NODE else self.ncell
        out = np.empty(n)
        check(sale_copy_field(self._h, name.encode(), out.ctypes.data_as(_dp), n))
        return out

    def set_field(self, name, values):
        a = np.ascontiguousarray(values, dtype=np.float64)
        check(sale_set_field(self._h, name.encode(), a.ctypes.data_as(_dp), a.size))

    def refresh(self):
        check(sale_refresh(self._h))

    def set_tiling(self, shape):
        check(sale_set_tiling(self._h, shape))

    def profile(self, on=True):
        check(sale_profile(self._h, 1 if on else 0))

    def profile_read(self, reset=True) -> dict:
        """{kernel name: (total ms, launches)} since the last reset."""
        n = sale_kernel_count()
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        check(sale_profile_read(self._h, ms, cnt, n, 1 if reset else 0))
        return {sale_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(n)}


class _Borrowed(State):
    """A mesh of a batch (the batch owns the handle and the memory)."""

    def __init__(self, handle, md, pd, stream):
        self._h = _vp(handle)
        self.md, self.pd, self.stream = md, pd, stream
        self.ncell, self.nnode = md.ncell, md.nnode

    def close(self):
        self._h = None


class Batch:
    """Independent meshes advanced together (FP32-mixed Eulerian cycle)."""

    def __init__(self, instances, device="cuda", stream=None):
        import torch

        self.instances = list(instances)
        n = len(self.instances)
        self._meshes = (sale_mesh_desc * n)(*[mesh_desc(md) for md, _ in self.instances])
        self._probs = (sale_problem_desc * n)(*[problem_desc(pd) for _, pd in self.instances])
        nbytes = sale_batch_bytes(n, self._meshes, SALE_FP32_MIXED)
        if nbytes == 0:
            raise SaleError(SALE_EINVAL, "bad batch description")
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self._h = _vp()
        check(sale_batch_create(n, self._meshes, self._probs, SALE_FP32_MIXED, _vp(self.buffer.data_ptr()),
                                nbytes, _vp(self.stream.cuda_stream), C.byref(self._h)))
        self.ncell_total = sum(md.ncell for md, _ in self.instances)

    def run(self, cycles):
        done = C.c_longlong(0)
        check(sale_batch_run(self._h, cycles, 1, C.byref(done)))
        return done.value

    def set_schedule(self, shape, order):
        check(sale_batch_set_schedule(self._h, shape, order))

    def state(self, i) -> State:
        md, pd = self.instances[i]
        return _Borrowed(sale_batch_state(self._h, i), md, pd, self.stream)

    def close(self):
        if getattr(self, "_h", None):
            sale_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
