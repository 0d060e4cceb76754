"""The FMA throughput probe the FP64 roofline is reported against.

sale_fma_probe must report an FP64 rate near the FP64 vector pipe's
nominal rate on GB300 (2 DFMA per clock per SM x 152 SMs x 2.07 GHz x 2
flop = 1.26 TFLOP/s; clocks may run lower under power management), an FP32
rate many times higher, and reject a buffer that is too small.
"""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2209_01983_gb300 import sale
    return sale, torch


def probe(sale, torch, precision, nbytes):
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    out = C.c_double(0.0)
    rc = sale.sale_fma_probe(precision, C.c_void_p(buf.data_ptr()), nbytes, C.c_void_p(st.cuda_stream),
                             C.byref(out))
    return rc, out.value


def test_fma_probe_rates(env):
    sale, torch = env
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rc, f64 = probe(sale, torch, sale.SALE_FP64, 8 * 256 * sms * 8)
    assert rc == sale.SALE_OK, sale.sale_last_error()
    nominal = 2 * sms * 2.07e9 * 2
    assert 0.5 * nominal <= f64 <= 1.1 * nominal, (f64, nominal)
    rc, f32 = probe(sale, torch, sale.SALE_FP32_MIXED, 8 * 256 * sms * 4)
    assert rc == sale.SALE_OK, sale.sale_last_error()
    assert f32 >= 10 * f64


def test_fma_probe_rejects_small_buffer(env):
    sale, torch = env
    rc, _ = probe(sale, torch, sale.SALE_FP64, 1024)
    assert rc == sale.SALE_ENOMEM
