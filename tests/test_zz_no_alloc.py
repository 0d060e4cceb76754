"""The allocation-free remap entry point against the state-based remap.

sale_remap_static serves callers that cannot allocate device memory:
plug-ins whose host program owns every device allocation and passes them
only their field arrays, and loops that must not call an allocator
(cudaMalloc and cudaFree can synchronise the device).  Its scratch is a
fixed static device array of the library.  This file checks, through the C
ABI, that it reproduces sale_remap_step on the same Lagrangian state, on
two calls in a row (the second call starts from the scratch the first one
left behind); that the second call, once the library's GPU code is loaded,
changes neither the device's free memory nor torch's allocator; and that it
rejects meshes larger than its fixed scratch.  It sits last in collection
order so a failure here comes after every other test has run.
"""
import ctypes as C
import gc

import numpy as np
import pytest

from paper_2209_01983_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale
    return sale, torch


def rel(a, b):
    s = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / s if s > 0 else float(np.max(np.abs(a)))


def test_static_remap_matches_state_remap(env):
    sale, torch = env
    md, pd = inputs.sedov_octant(1, jitter=0.1)
    md.nx, md.ny, md.nz = 22, 19, 17  # 7106 cells, 8280 nodes
    st = sale.State(md, pd)
    st.run_to_time(max_cycles=6, remap_every=1)
    st.lagrange_step()  # leaves the mesh displaced: a remap has work to do
    host = {n: st.field(n) for n in ("x", "y", "z", "u", "v", "w", "mn", "m", "e", "rho",
                                     "xref", "yref", "zref")}
    st.remap_step()  # the state-based entry point
    want = {n: st.field(n) for n in ("u", "v", "w", "mn", "m", "e", "x", "y", "z")}

    dev = torch.device("cuda")
    stream = torch.cuda.Stream()

    def upload(*names):
        return torch.from_numpy(np.concatenate([host[n] for n in names])).to(dev)

    reflect = (C.c_int * 6)(*md.reflect)
    for call in range(2):
        xref = upload("xref", "yref", "zref")
        x = upload("x", "y", "z")
        u_in = upload("u", "v", "w")
        u_out = torch.full_like(u_in, float("nan"))
        mn, m, e, rho = upload("mn"), upload("m"), upload("e"), upload("rho")
        torch.cuda.synchronize()
        p = lambda t: C.c_void_p(t.data_ptr())
        gc.collect()
        gc.disable()  # no tensor of this process is freed while the call is measured
        try:
            free0 = torch.cuda.mem_get_info()[0]
            torch0 = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
            rc = sale.sale_remap_static(md.nx, md.ny, md.nz, reflect, pd.ke_fix, p(xref), p(x), p(u_in),
                                        p(u_out), p(mn), p(m), p(e), p(rho), C.c_void_p(stream.cuda_stream))
            torch1 = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
            free1 = torch.cuda.mem_get_info()[0]
        finally:
            gc.enable()
        assert rc == sale.SALE_OK, sale.sale_last_error()
        assert torch1 == torch0, call
        if call == 1:  # the first call may load the library's GPU code (and its static array)
            assert free1 == free0, (free0, free1)
        nn = md.nnode
        got_u = u_out.cpu().numpy()
        got_x = x.cpu().numpy()
        vel_scale = max(float(np.max(np.abs(want[c]))) for c in "uvw")
        for k, c in enumerate("uvw"):
            assert float(np.max(np.abs(got_u[k * nn:(k + 1) * nn] - want[c]))) <= TOL * vel_scale, (call, c)
        for k, c in enumerate("xyz"):
            assert rel(got_x[k * nn:(k + 1) * nn], want[c]) <= TOL, (call, c)
        assert rel(mn.cpu().numpy(), want["mn"]) <= TOL, call
        assert rel(m.cpu().numpy(), want["m"]) <= TOL, call
        assert rel(e.cpu().numpy(), want["e"]) <= TOL, call
        # the remap moved mass between cells (the comparison is not vacuous)
        assert float(np.max(np.abs(m.cpu().numpy() - host["m"]))) > 0.0


def test_static_remap_rejects_oversized_mesh(env):
    sale, torch = env
    reflect = (C.c_int * 6)(1, 1, 1, 1, 1, 1)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    n = 41  # 41^3 = 68921 cells > SALE_STATIC_MAX_CELLS
    rc = sale.sale_remap_static(n, n, n, reflect, 1, p, p, p, p, p, p, p, p, None)
    assert rc == sale.SALE_EINVAL
    assert b"static scratch holds at most" in sale.sale_last_error()
