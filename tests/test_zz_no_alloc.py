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


def _call(L, scene, image, records, moments, stream, first=None):
    u64p = C.POINTER(C.c_uint64)
    fst = None if first is None else np.ascontiguousarray(first, np.uint64)
    return L.phosim_trace_noalloc(scene.h, scene.src, len(scene.sources), scene.n_photons.ctypes.data_as(u64p),
                                  None if fst is None else fst.ctypes.data_as(u64p),
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
    # host records or moments are refused before anything is launched (the kernels would write through them)
    assert _call(L, s, img, torch.zeros(8, dtype=torch.uint8), mom, stream) == -1
    assert _call(L, s, img, rec, torch.zeros((1, P.MOMENT_WORDS), dtype=torch.float64), stream) == -1
    s.close()


def test_noalloc_refuses_a_capturing_stream():
    """The call copies its source list from host memory it frees on return, so on a stream that is being
    captured it returns INVALID_ARGUMENT and records nothing; after the capture it runs as before."""
    L = P.lib()
    L.phosim_trace_noalloc.argtypes = [C.c_void_p, C.POINTER(P.Source), C.c_int, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    counts = [500, 700]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=17))
    ref = G.run_gpu(sc, P.PLAIN_FP64)
    s = P.Scene(sc, P.PLAIN_FP64)
    d = sc.detector
    n = int(np.sum(counts))
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
    # set-up (the scratch address lookup) happens on the first call, before the capture
    assert _call(L, s, img, rec, mom, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            rc = _call(L, s, img, rec, mom, side.cuda_stream)
        finally:
            g.capture_end()
    assert rc == -1
    torch.cuda.synchronize()
    img.zero_(); rec.zero_(); mom.zero_()
    assert _call(L, s, img, rec, mom, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy().view(np.uint32), ref["image"])
    assert np.array_equal(P.records_to_numpy(rec), ref["rec"])
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


def test_noalloc_double_single_with_bundles_and_photon_offsets():
    """Double-single with a background source traced as rays of 8 photons and nonzero first photon indices:
    the one-kernel form (photon units) and phosim_trace's two-kernel form (ray units, the bundle stage) give the
    same records and image for the same photon ranges."""
    from paper_1504_06570_gb300 import inputs as I
    L = P.lib()
    L.phosim_trace_noalloc.argtypes = [C.c_void_p, C.POINTER(P.Source), C.c_int, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    counts = [1000, 3000, 4000]
    src = G.mixed_sources(counts, seed=19)
    src.kind[2] = I.GAUSS
    src.a[2] = 2e-5
    src.bundle = np.array([1, 1, 8], np.int32)
    src.bundle_sigma = np.array([0.0, 0.0, 0.004])
    sc = G.test_system_scene(sources=src)
    first = np.array([5, 123456, 8 * 1000 + 3], np.uint64)      # the last starts 3 photons into a ray
    n = int(np.sum(counts))
    ref = G.run_gpu(sc, P.MIXED_DS, early_reject=True, first=first)
    s = P.Scene(sc, P.MIXED_DS, early_reject=True)
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
    assert _call(L, s, img, rec, mom, torch.cuda.current_stream().cuda_stream, first=first) == 0
    torch.cuda.synchronize()
    r = P.records_to_numpy(rec)
    assert np.array_equal(r, ref["rec"])
    assert np.array_equal(img.cpu().numpy().view(np.uint32), ref["image"])
    assert (r["flags"][4000:] & 1).sum() > 100           # the bundled source reaches the chip
    np.testing.assert_allclose(mom.cpu().numpy(), ref["moments"], rtol=1e-5, atol=1e-6)
    s.close()
