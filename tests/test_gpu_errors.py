"""Error paths through the C ABI on a device: malformed descriptors return error codes and leave the scene
usable; per-photon failures (a ray outside a surface's domain) are flags and counters, never faults."""
import ctypes as C

import numpy as np
import pytest

from paper_1504_06570_gb300 import inputs as I
from paper_1504_06570_gb300 import phosim as P
from tests import gpu_helpers as G
from tests.helpers import bare_scene

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_load_errors_leave_the_scene_usable():
    sc = I.paraboloid_scene(n_photons=2000, screen_n=128)
    s = P.Scene(sc)
    L = s.L
    # detector not last
    bad = [I.Surface(kind=I.DETECTOR, z=10000.0, material=1), I.Surface(kind=I.MIRROR, R=20000.0, kappa=-1.0)]
    with pytest.raises(P.PhosimError) as e:
        s.load_optics(bad, sc.materials, [])
    assert e.value.code == -1
    # too many surfaces
    with pytest.raises(P.PhosimError) as e:
        s.load_optics([I.Surface(kind=I.REFRACT, z=float(i)) for i in range(16)] + [I.Surface(kind=I.DETECTOR)],
                      sc.materials, [])
    assert e.value.code == -6
    # layers not top to bottom
    ph = np.zeros((8, 8))
    with pytest.raises(P.PhosimError) as e:
        s.load_screens([I.Layer(z=1e6, scales=[I.ScreenScale(10.0, ph)]), I.Layer(z=2e6, scales=[I.ScreenScale(10.0, ph)])])
    assert e.value.code == -1
    # negative flux
    flux = -np.ones((1, 10))
    assert L.phosim_load_seds(s.h, flux.ctypes.data_as(C.POINTER(C.c_double)), 1, 10, 400.0, 1.0) == -1
    # gradient parameter field out of range
    with pytest.raises(P.PhosimError) as e:
        s.grad(np.zeros((1, 5)), [(0, 7)])
    assert e.value.code == -1
    # the scene still traces exactly as a fresh one
    ref = G.run_gpu(sc, P.PLAIN_FP64, records=False)
    img = torch.zeros((256, 256), dtype=torch.int32, device="cuda")
    s.trace(img)
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy().view(np.uint32), ref["image"])
    s.close()


def test_trace_before_loading_is_not_ready():
    sc = I.paraboloid_scene(n_photons=10, screen_n=64)
    d = sc.detector
    ell, sig = np.ascontiguousarray(d.ell), np.ascontiguousarray(d.sigma)
    desc = P.SceneDesc(seed=1, precision=0, flags=0, pupil_r_in=0.0, pupil_r_out=500.0, h_top=1e8, z_entrance=11000.0,
                       lambda_ref=500.0, nx=16, ny=16, pixel=0.01, t_si=0.1, ell_lam0=d.ell_lam0, ell_dlam=1.0,
                       n_ell=len(ell), ell=ell.ctypes.data_as(C.POINTER(C.c_double)), n_sigma=2,
                       sigma=sig.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    L = P.lib()
    assert L.phosim_create_scene(C.byref(desc), C.byref(h)) == 0
    src = P.sources_struct(sc.sources)
    cnt = np.array([10], np.uint64)
    img = torch.zeros((16, 16), dtype=torch.int32, device="cuda")
    rc = L.phosim_trace(h, src, 1, cnt.ctypes.data_as(C.POINTER(C.c_uint64)), None, C.c_void_p(img.data_ptr()),
                        None, None, None)
    assert rc == -5
    L.phosim_destroy_scene(h)


def test_rays_outside_a_surface_domain_are_flagged(oracle_mod):
    """A sphere of radius 600 mm lit over 700 mm: rays beyond r = R have no intersection with its vertex
    branch and are dropped as MISSED, identically in the oracle and the kernel."""
    surfaces = [I.Surface(kind=I.MIRROR, R=600.0, kappa=0.0, z=0.0, r_out=700.0),
                I.Surface(kind=I.DETECTOR, z=300.0, material=1)]
    sc = bare_scene(surfaces, n_photons=20000, pupil=(0.0, 700.0), nx=2048, pixel=0.5)
    gpu = G.run_gpu(sc, P.PLAIN_FP64)
    ora = G.oracle_trace(oracle_mod, sc)
    reason_g = (gpu["rec"]["flags"] >> 8) & 0xFF
    reason_o = (ora["flags"] >> 8) & 0xFF
    assert (reason_o == 2).sum() > 1000
    assert np.array_equal(reason_g == 2, reason_o == 2)
    assert gpu["counters"][1 + 2] == (reason_g == 2).sum()


def test_newton_iteration_cap_is_a_flag_not_a_fault():
    """A flat plate carrying a steep 10th-order asphere (alpha_10 r^10 reaches kilometres at the rim) seen by
    tilted rays: Newton's method from the plane's root cannot converge within the iteration cap for many rays.
    They are dropped as NEWTON and counted; the launch completes and the context stays usable."""
    surfaces = [I.Surface(kind=I.REFRACT, R=0.0, alpha=(0, 0, 0, 0, 0, 0, 0, 1e-20), z=0.0, r_out=500.0, material=0),
                I.Surface(kind=I.DETECTOR, z=-1000.0, material=1)]
    src = I.point_sources([0.3], [0.0], [5000])
    sc = bare_scene(surfaces, n_photons=5000, pupil=(0.0, 500.0), nx=4096, pixel=1.0, sources=src)
    sc.z_entrance = 2.0e7
    gpu = G.run_gpu(sc, P.PLAIN_FP64)
    reasons = (gpu["rec"]["flags"] >> 8) & 0xFF
    assert (reasons == 3).sum() > 0
    assert gpu["counters"][1 + 3] == (reasons == 3).sum()
    again = G.run_gpu(I.paraboloid_scene(n_photons=1000, screen_n=64), P.PLAIN_FP64, records=False)
    assert again["counters"][0] == 1000


def test_grad_refuses_ghosts():
    """The adjoint follows forward paths only: a scene whose coatings reflect is UNSUPPORTED for phosim_grad."""
    from tests import gpu_helpers as GH
    sc = GH.test_system_scene(n_photons=100, atmosphere=False)
    sc.coatings[0].reflect = 0.5 * (1.0 - sc.coatings[0].table)
    s = P.Scene(sc)
    with pytest.raises(P.PhosimError) as e:
        s.grad(np.zeros((1, 5)), [(0, 0)])
    assert e.value.code == -4
    s.close()


def test_stage_timing_reports_each_kernel():
    """phosim_set_stage_timing / phosim_stage_times: the double-single trace launches the chief-ray, entry and
    optics kernels, whose event times are positive and add up to the call's own time; a short output array is
    refused."""
    import ctypes as C
    sc = I.paraboloid_scene(n_photons=200_000, screen_n=128)
    s = P.Scene(sc, P.MIXED_DS, early_reject=True)
    L = P.lib()
    img = torch.zeros((256, 256), dtype=torch.int32, device="cuda")
    assert L.phosim_set_stage_timing(s.h, 1) == 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    s.trace(img)
    b.record()
    ms = (C.c_double * 5)()
    assert L.phosim_stage_times(s.h, ms, 5) == 0
    torch.cuda.synchronize()
    t = list(ms)
    assert t[0] > 0 and t[1] == 0 and t[2] > 0 and t[3] > 0 and t[4] == 0
    assert sum(t) <= a.elapsed_time(b) * 1.05 + 0.05
    assert L.phosim_stage_times(s.h, ms, 4) == -1
    L.phosim_set_stage_timing(s.h, 0)
    s.close()


def test_bundle_and_reflection_limits():
    """Background bundles above PHOSIM_MAX_BUNDLE are LIMIT, negative ones or a negative spread INVALID; a
    reflection table with T + R > 1 or R < 0 is refused at load; the scene stays usable."""
    sc = I.paraboloid_scene(n_photons=1000, screen_n=64)
    s = P.Scene(sc)
    img = torch.zeros((256, 256), dtype=torch.int32, device="cuda")
    for bundle, sigma, code in ((4097, 0.01, -6), (-1, 0.01, -1), (8, -0.5, -1)):
        src = sc.sources.subset([0])
        src.bundle = np.array([bundle], np.int32)
        src.bundle_sigma = np.array([sigma])
        s.set_sources(src)
        with pytest.raises(P.PhosimError) as e:
            s.trace(img)
        assert e.value.code == code, (bundle, sigma)
    s.set_sources(sc.sources)
    for R in (0.6, -0.1):
        coat = I.Coating(lam0=400.0, dlam=300.0, theta0=0.0, dtheta=1.6, table=np.array([[0.5]]),
                         reflect=np.array([[R]]))
        with pytest.raises(P.PhosimError) as e:
            s.load_optics(sc.surfaces, sc.materials, [coat])
        assert e.value.code == -1
    ref = G.run_gpu(sc, P.PLAIN_FP64, records=False)
    img.zero_()
    s.trace(img)
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy().view(np.uint32), ref["image"])
    s.close()


def test_host_records_or_moments_are_refused_before_launch():
    """phosim_trace writes records and moment sums from its kernels, so they must be device memory of the
    scene's device: host tensors return INVALID_ARGUMENT and nothing is launched (the image is untouched)."""
    sc = G.test_system_scene(sources=G.mixed_sources([300, 200]))
    for prec in (P.PLAIN_FP64, P.MIXED_DS):
        s = P.Scene(sc, prec)
        d = sc.detector
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        rec_dev = torch.zeros(500 * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        mom_dev = torch.zeros((2, P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
        for rec, mom in ((torch.zeros(500 * P.RECORD_DTYPE.itemsize, dtype=torch.uint8), mom_dev),
                         (rec_dev, torch.zeros((2, P.MOMENT_WORDS), dtype=torch.float64)),
                         (torch.zeros(500 * P.RECORD_DTYPE.itemsize, dtype=torch.uint8).pin_memory(), None)):
            with pytest.raises(P.PhosimError) as e:
                s.trace(img, rec, mom)
            assert e.value.code == -1
        torch.cuda.synchronize()
        assert int(img.sum()) == 0
        s.trace(img, rec_dev, mom_dev)
        torch.cuda.synchronize()
        assert int(img.sum()) > 0
        s.close()


def test_autotune_keeps_a_listed_candidate_and_results_do_not_change():
    """phosim_autotune times each candidate launch shape on a sample of the workload and keeps the fastest:
    the scene then reports one of the listed candidates (phosim_get_schedule), and traces give bit-identical
    records and image before and after (the random numbers are counter-based), and the same moment sums up to
    their summation order."""
    counts = [5000, 20000, 1, 0, 7000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=23))
    for prec in (P.PLAIN_FP64, P.MIXED_DS):
        before = G.run_gpu(sc, prec, early_reject=True)
        s = P.Scene(sc, prec, early_reject=True)
        assert s.schedule() == (256, 0)
        t, k = s.autotune(sample_photons=20000)
        assert t in (64, 128, 256) and k in (64, 256, 1024, 4096)
        assert s.schedule() == (t, k)
        n = int(np.sum(counts))
        d = sc.detector
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
        s.trace(img, rec, mom)
        torch.cuda.synchronize()
        assert np.array_equal(P.records_to_numpy(rec), before["rec"])
        assert np.array_equal(img.cpu().numpy().view(np.uint32), before["image"])
        # sums are reduced per tile before atomics, so their rounding order follows the schedule
        np.testing.assert_allclose(mom.cpu().numpy(), before["moments"], rtol=1e-10, atol=1e-10)
        # every other listed schedule gives the same records too
        for tt, kk in ((64, 64), (128, 4096)):
            s.set_schedule(tt, kk)
            assert s.schedule() == (tt, kk)
            rec.zero_()
            img.zero_()
            s.trace(img, rec, None)
            torch.cuda.synchronize()
            assert np.array_equal(P.records_to_numpy(rec), before["rec"])
        s.close()


def test_moments_derive_matches_two_pass_moments_of_the_records():
    """phosim_moments_derive turns the additive sums into the count, centroid and central second moments;
    they equal the two-pass moments of the detected records' positions (FP64 path)."""
    counts = [3000, 500, 0]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=29))
    out = G.run_gpu(sc, P.PLAIN_FP64)
    m = P.derived_moments(out["moments"])
    r = out["rec"]
    src = np.repeat(np.arange(len(counts)), counts)
    for s_ in range(2):
        k = (src == s_) & ((r["flags"] & 1) == 1)
        x, y = r["x"][k], r["y"][k]
        exp = [k.sum(), x.mean(), y.mean(), ((x - x.mean()) ** 2).mean(), ((x - x.mean()) * (y - y.mean())).mean(),
               ((y - y.mean()) ** 2).mean()]
        np.testing.assert_allclose(m[s_], exp, rtol=1e-9, atol=1e-12)
    assert m[2, 0] == 0 and np.all(np.isnan(m[2, 1:]))
