"""The measurement probes of phosim_bench.h on a device: the FMA, double-single and random-gather rates that
the benchmark's rooflines divide by are positive, ordered as the hardware orders them, and argument errors
are reported before anything runs."""
import ctypes as C

import pytest

from paper_1504_06570_gb300 import phosim as P

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

INVALID_ARGUMENT = -1        # PHOSIM_ERR_INVALID_ARGUMENT


def _lib():
    return P.lib()


def test_fma_and_double_single_rates():
    L = _lib()
    r = C.c_double()
    assert L.phosim_fma_rate(0, 2000, 4, None, C.byref(r)) == 0
    fp32 = r.value
    assert L.phosim_fma_rate(1, 200, 4, None, C.byref(r)) == 0
    fp64 = r.value
    assert fp32 > 10 * fp64 > 0
    rates = []
    for op in range(5):
        assert L.phosim_ds_rate(op, 500, 4, None, C.byref(r)) == 0
        rates.append(r.value)
    # a double-single sum or product is several FP32 instructions; the quotient and root more again
    assert all(0 < x < fp32 / 2 for x in rates)
    assert min(rates[0], rates[1]) > max(rates[3], rates[4])
    assert L.phosim_ds_rate(5, 500, 4, None, C.byref(r)) == INVALID_ARGUMENT


def test_random_gather_rates():
    """32-byte gathers from a buffer well inside the L2 run faster than from one far larger than it, and both
    stay below a plausible ceiling for the bytes they gather."""
    L = _lib()
    r = C.c_double()
    assert L.phosim_gather_rate(C.c_size_t(1 << 30), 512, 4, None, C.byref(r)) == 0
    hbm = r.value
    assert L.phosim_gather_rate(C.c_size_t(16 << 20), 512, 4, None, C.byref(r)) == 0
    l2 = r.value
    assert 0 < hbm < l2 < 1e5, (hbm, l2)
    for bad in (0, 1000, (1 << 20) + 8, 1 << 40):
        assert L.phosim_gather_rate(C.c_size_t(bad), 512, 4, None, C.byref(r)) == INVALID_ARGUMENT
    assert L.phosim_gather_rate(C.c_size_t(1 << 20), 0, 4, None, C.byref(r)) == INVALID_ARGUMENT
