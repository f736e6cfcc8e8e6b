"""The allocation-free trace entry point, for callers of this library that cannot call cudaMalloc (their
device memory belongs to an outside pool, or an allocation would synchronise the device in a
latency-critical loop).  Through the C ABI, two calls in a row must give exactly what phosim_trace gives
(same kernels, same photons): images, moment sums and per-photon records.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_1504_06570_gb300 import phosim as P
from tests import gpu_helpers as G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _call(L, scene, image, records, moments, stream):
    u64p = C.POINTER(C.c_uint64)
    return L.phosim_trace_noalloc(scene.h, scene.src, len(scene.sources), scene.n_photons.ctypes.data_as(u64p), None,
                                  C.c_void_p(image.data_ptr()), C.c_void_p(records.data_ptr()),
                                  C.c_void_p(moments.data_ptr()), C.c_void_p(stream))


def test_noalloc_matches_trace_twice_in_a_row():
    from paper_1504_06570_gb300 import build
    build.build()
    L = P.lib()
    L.phosim_trace_noalloc.argtypes = [C.c_void_p, C.POINTER(P.Source), C.c_int, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    counts = [0, 1, 31, 33, 1000, 4097, 3000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=11))
    n = int(np.sum(counts))
    ref = G.run_gpu(sc, P.PLAIN_FP64)
    s = P.Scene(sc, P.PLAIN_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    d = sc.detector
    for _ in range(2):
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
        assert _call(L, s, img, rec, mom, stream) == 0
        torch.cuda.synchronize()
        assert np.array_equal(img.cpu().numpy().view(np.uint32), ref["image"])
        assert np.array_equal(P.records_to_numpy(rec), ref["rec"])
        np.testing.assert_allclose(mom.cpu().numpy(), ref["moments"], rtol=1e-12, atol=1e-15)
    # sizes beyond the documented maximum and host images are refused
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    rec = torch.zeros(8, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((1, P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
    too_many = (P.Source * 4097)()
    cnt = np.ones(4097, np.uint64)
    rc = L.phosim_trace_noalloc(s.h, too_many, 4097, cnt.ctypes.data_as(C.POINTER(C.c_uint64)), None,
                                C.c_void_p(img.data_ptr()), None, None, C.c_void_p(stream))
    assert rc == -6
    host = torch.zeros((d.ny, d.nx), dtype=torch.int32)
    assert _call(L, s, host, rec, mom, stream) == -1
    s.close()


def test_noalloc_double_single_matches_two_kernel_trace():
    """In the double-single precision the allocation-free entry runs the one-kernel form of the path and
    phosim_trace the two-kernel form (entry stage, states in device memory, optics stage): the same
    per-photon arithmetic, so identical records and images; the moment sums differ only by the order of the
    single-precision partial sums."""
    L = P.lib()
    L.phosim_trace_noalloc.argtypes = [C.c_void_p, C.POINTER(P.Source), C.c_int, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    counts = [0, 1, 31, 33, 1000, 4097, 3000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=13), hf=True)
    n = int(np.sum(counts))
    ref = G.run_gpu(sc, P.MIXED_DS, early_reject=True)
    s = P.Scene(sc, P.MIXED_DS, early_reject=True)
    stream = torch.cuda.current_stream().cuda_stream
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
    assert _call(L, s, img, rec, mom, stream) == 0
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy().view(np.uint32), ref["image"])
    assert np.array_equal(P.records_to_numpy(rec), ref["rec"])
    np.testing.assert_allclose(mom.cpu().numpy(), ref["moments"], rtol=1e-5, atol=1e-6)
    s.close()
