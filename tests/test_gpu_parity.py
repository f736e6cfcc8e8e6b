"""Parity of the CUDA path (through the C ABI) with the CPU oracle, photon by photon, on seeded inputs.

Tolerances (written from the arithmetic): the FP64 path and the oracle evaluate the same formulas with
different operation order and contraction, so final positions agree to ~1e-12 mm; the per-photon gate is
1e-4 pixel for at least 99.999 % of the photons detected by both, with identical fates
except for photons within 1e-7 mm / 1e-6 nm of an accept boundary.  The mixed path keeps positions and
intersections in FP64 and rounds the deflections, the wavelength blur and the sensor draws to FP32, so it
is held to the moment gate (0.1 %) and to 1e-2 pixel per photon for 99.9 % of the photons.  The
double-single path (MIXED_DS) keeps the same parts at about 48 significant bits instead of 53 and is held to
the mixed path's gates everywhere, and to the FP64 per-photon gate where no single-precision step is on the
path (atmosphere and sensor off).
"""
import numpy as np
import pytest

from paper_1504_06570_gb300 import inputs as I
from paper_1504_06570_gb300 import phosim as P
from tests import gpu_helpers as G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1504_06570_gb300 import build
    build.build()


def test_tiny_paraboloid_fp64_per_photon(oracle_mod):
    """1 on-axis star, 1e5 photons, 5800 K blackbody 400-700 nm, one 512^2 Kolmogorov screen at 5 km,
    D = 1 m f/10 paraboloid, 256^2 chip of 10 um pixels with 100 um of silicon, FP64 throughout."""
    sc = I.paraboloid_scene(n_photons=100_000)
    gpu = G.run_gpu(sc, P.PLAIN_FP64)
    ora = G.oracle_trace(oracle_mod, sc)
    r = G.compare_records(sc, gpu, ora, pos_tol_px=1e-4, min_frac=0.99999)
    assert r["max_err_px"] < 1e-6, r
    assert r["lam_err"] < 1e-9
    # the image is the histogram of the records' pixels, and the oracle's image away from boundaries
    assert np.array_equal(gpu["image"], G.image_from_pix(gpu["rec"], sc.detector))
    diff = np.abs(gpu["image"].astype(np.int64) - ora["image"].astype(np.int64)).sum()
    assert diff <= 2 * r["n_boundary"]
    G.compare_moments(gpu["moments"], G.oracle_moments(ora, 1), rel=1e-6)
    c = gpu["counters"]
    assert c[0] == 100_000 and c[1] == ((ora["flags"] & 1) == 1).sum()
    assert c[0] == c[1] + c[2:].sum()


@pytest.mark.parametrize("precision", [P.MIXED, P.MIXED_DS])
def test_tiny_paraboloid_mixed(oracle_mod, precision):
    sc = I.paraboloid_scene(n_photons=100_000)
    gpu = G.run_gpu(sc, precision)
    ora = G.oracle_trace(oracle_mod, sc)
    rec = gpu["rec"]
    both = ((rec["flags"] & 1) == 1) & ((ora["flags"] & 1) == 1)
    err = np.hypot(rec["x"][both] - ora["x"][both], rec["y"][both] - ora["y"][both]) / sc.detector.pixel
    assert np.mean(err < 1e-2) > 0.999, np.percentile(err, [50, 99, 99.9, 100])
    assert np.mean(rec["flags"] != ora["flags"]) < 1e-3
    G.compare_moments(gpu["moments"], G.oracle_moments(ora, 1), rel=1e-3)


def test_double_single_fates_and_moments_at_fp64_level(oracle_mod):
    """The double-single path's coating decisions use its double-single wavelength (the FP64 paths' bins), so
    with the atmosphere, the sensor, every source kind and the dynamic transmission test on it gives every photon
    the oracle's fate except at flagged accept boundaries, and its moments agree with the oracle far inside the
    mixed gate: centroids within 1e-5 of the PSF size and second moments within 1e-5 relative (the remaining
    differences are the single-precision deflections, diffusion draws and wavelength of the FP32 steps)."""
    counts = [0, 1, 31, 33, 1000, 4097, 20000, 7, 2500]
    sc = G.test_system_scene(sources=G.mixed_sources(counts), hf=True)
    gpu = G.run_gpu(sc, P.MIXED_DS)
    ora = G.oracle_trace(oracle_mod, sc)
    rec = gpu["rec"]
    bnd = G.boundary_mask(ora)
    assert np.all((rec["flags"] == ora["flags"]) | bnd), np.sum((rec["flags"] != ora["flags"]) & ~bnd)
    G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-5)
    both = ((rec["flags"] & 1) == 1) & ((ora["flags"] & 1) == 1)
    err = np.maximum(np.abs(rec["x"][both] - ora["x"][both]), np.abs(rec["y"][both] - ora["y"][both])) / sc.detector.pixel
    assert np.percentile(err, 99.9) < 1e-3, np.percentile(err, [50, 99.9, 100])
    assert np.max(np.abs(rec["lam"] - ora["lam"]) / ora["lam"]) < 1e-7


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_catadioptric_system_all_surface_features(oracle_mod, precision):
    """Annular paraboloid with Zernike figure and tilt, decentred aspheric lens, coated filter, silicon;
    two layers of two scales with wind; point, Sersic and Gaussian sources with redshifts; ragged counts."""
    counts = [0, 1, 31, 33, 1000, 4097, 20000, 7, 2500]
    sc = G.test_system_scene(sources=G.mixed_sources(counts))
    gpu = G.run_gpu(sc, precision)
    ora = G.oracle_trace(oracle_mod, sc)
    if precision == P.PLAIN_FP64:
        r = G.compare_records(sc, gpu, ora)
        assert r["max_err_px"] < 1e-6, r
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-6)
    else:
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-3)
    assert np.array_equal(gpu["image"], G.image_from_pix(gpu["rec"], sc.detector))


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_second_atmospheric_kick(oracle_mod, precision):
    """Sec. 2.3.2 second kick: the same scene with the high-frequency kick table loaded."""
    counts = [4000, 2500, 33]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=8), hf=True)
    gpu = G.run_gpu(sc, precision, early_reject=True)
    ora = G.oracle_trace(oracle_mod, sc)
    det_g, det_o = (gpu["rec"]["flags"] & 1) == 1, (ora["flags"] & 1) == 1
    if precision == P.PLAIN_FP64:
        assert np.all((det_g == det_o) | G.boundary_mask(ora))
        both = det_g & det_o
        err = np.maximum(np.abs(gpu["rec"]["x"][both] - ora["x"][both]), np.abs(gpu["rec"]["y"][both] - ora["y"][both]))
        assert err.max() / sc.detector.pixel < 1e-6
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-6)
    else:
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-3)


@pytest.mark.parametrize("schedule", [(32, 32), (64, 96), (256, 1024), (128, 0)])
def test_schedule_does_not_change_results(oracle_mod, schedule):
    """Counter-based streams: the result depends on neither the block size nor the tile size."""
    counts = [3, 500, 1200, 64]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=9))
    ref = G.run_gpu(sc, P.PLAIN_FP64)
    gpu = G.run_gpu(sc, P.PLAIN_FP64, schedule=schedule)
    assert np.array_equal(gpu["rec"], ref["rec"])
    assert np.array_equal(gpu["image"], ref["image"])


@pytest.mark.parametrize("schedule", [(32, 32), (64, 96), (128, 0), (256, 1024)])
def test_schedule_does_not_change_double_single_stages(schedule):
    """The two-kernel double-single path (entry, optics and bundle stages, each with its own grid) under any
    block and tile size: every photon is accounted for once and the records and image do not change."""
    counts = [3, 5000, 12000, 640, 2000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=19))
    sc.sources.bundle = np.array([1, 1, 1, 1, 8], np.int32)
    sc.sources.bundle_sigma = np.array([0.0, 0.0, 0.0, 0.0, 0.004])
    ref = G.run_gpu(sc, P.MIXED_DS, early_reject=True)
    gpu = G.run_gpu(sc, P.MIXED_DS, early_reject=True, schedule=schedule)
    n = int(np.sum(counts))
    for out in (ref, gpu):
        c = out["counters"]
        assert c[0] == n and c[1] + sum(c[2:]) == n, c
        assert np.count_nonzero(out["rec"]["flags"]) == n
    assert np.array_equal(gpu["rec"], ref["rec"])
    assert np.array_equal(gpu["image"], ref["image"])


def test_photon_ranges_compose():
    """Tracing photons [0, a) then [a, n) of each source gives the records and image of [0, n)."""
    counts = np.array([700, 1500, 33], np.uint64)
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=4))
    full = G.run_gpu(sc, P.PLAIN_FP64)
    a = np.array([300, 1, 32], np.uint64)
    p1 = G.run_gpu(sc, P.PLAIN_FP64, n_photons=a)
    p2 = G.run_gpu(sc, P.PLAIN_FP64, n_photons=counts - a, first=a)
    assert np.array_equal(p1["image"] + p2["image"], full["image"])
    off = np.r_[0, np.cumsum(counts)]
    o1, o2 = np.r_[0, np.cumsum(a)], np.r_[0, np.cumsum(counts - a)]
    for s in range(3):
        joined = np.concatenate([p1["rec"][o1[s]:o1[s + 1]], p2["rec"][o2[s]:o2[s + 1]]])
        assert np.array_equal(joined, full["rec"][off[s]:off[s + 1]])


def test_host_image_is_staged():
    sc = I.paraboloid_scene(n_photons=20000)
    dev = G.run_gpu(sc, P.PLAIN_FP64, records=False)
    host = G.run_gpu(sc, P.PLAIN_FP64, records=False, host_image=True)
    assert np.array_equal(dev["image"], host["image"])


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED_DS])
def test_sensor_off_and_atmosphere_off(oracle_mod, precision):
    """Without the atmosphere and the sensor, only the wavelength blur is single precision in the
    double-single path (24 of the draw's 32 bits, about 1e-7 nm): it meets the FP64 per-photon gate."""
    sc = G.test_system_scene(n_photons=20000, sensor=False, atmosphere=False)
    gpu = G.run_gpu(sc, precision)
    ora = G.oracle_trace(oracle_mod, sc)
    r = G.compare_records(sc, gpu, ora)
    assert r["max_err_px"] < (1e-6 if precision == P.PLAIN_FP64 else 1e-4), r


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_early_rejection_keeps_the_detected_photons(oracle_mod, precision):
    """Dynamic transmission (Sec. 3.2): deciding the coating draws up front changes only the reported reason
    of photons lost anyway; detected photons, image and moments are those of the full trace."""
    counts = [5000, 700, 12000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=5))
    full = G.run_gpu(sc, precision)
    early = G.run_gpu(sc, precision, early_reject=True)
    det_f = (full["rec"]["flags"] & 1) == 1
    det_e = (early["rec"]["flags"] & 1) == 1
    assert np.array_equal(det_f, det_e)
    assert np.array_equal(full["rec"][det_f], early["rec"][det_e])
    assert np.array_equal(full["image"], early["image"])
    np.testing.assert_allclose(early["moments"], full["moments"], rtol=1e-12, atol=1e-15)
    moved = (~det_e) & (full["rec"]["flags"] != early["rec"]["flags"])
    assert np.all(((early["rec"]["flags"][moved] >> 8) & 0xFF) == 5)
    if precision == P.PLAIN_FP64:
        ora = G.oracle_trace(oracle_mod, sc)
        assert np.array_equal(det_e, (ora["flags"] & 1) == 1)


@pytest.mark.parametrize("precision", [P.MIXED, P.MIXED_DS])
def test_graph_replay_matches_direct_launches(precision):
    """PHOSIM_GRAPH: the captured launch pair replays with each call's parameters (different photon ranges,
    a different source count) and gives the direct launches' records and images."""
    import torch
    counts = np.array([700, 1500, 33], np.uint64)
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=4))
    ref = P.Scene(sc, precision, early_reject=True)
    gr = P.Scene(sc, precision, early_reject=True, graph=True)
    d = sc.detector
    for first, sub in ((None, None), (np.array([5, 0, 1], np.uint64), None), (None, [1])):
        outs = []
        for s in (ref, gr):
            if sub is not None:
                s.set_sources(sc.sources.subset(sub))
            n = int(s.n_photons.sum())
            img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
            rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            s.trace(img, rec, None, first=first)
            torch.cuda.synchronize()
            outs.append((img.cpu().numpy(), P.records_to_numpy(rec)))
        assert np.array_equal(outs[0][0], outs[1][0])
        assert np.array_equal(outs[0][1], outs[1][1])
    ref.close()
    gr.close()


def test_graph_follows_the_kernel_list():
    """In the double-single path the captured graph holds 3 to 5 kernels (chief rays, entry and optics stages,
    the bundle stage when a source is bundled, the moment-stripe sum when moment sums are asked for); a scene
    that alternates between those lists in graph mode re-captures and gives, every time, the images, records and
    moment sums of the same calls launched directly."""
    import torch
    counts = np.array([900, 2500, 60], np.uint64)
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=31))
    bundled = G.test_system_scene(sources=G.mixed_sources(counts, seed=31))
    bundled.sources.bundle = np.array([1, 4, 1], np.int32)
    bundled.sources.bundle_sigma = np.array([0.0, 0.003, 0.0])
    ref = P.Scene(sc, P.MIXED_DS, early_reject=True)
    gr = P.Scene(sc, P.MIXED_DS, early_reject=True, graph=True)
    d = sc.detector
    n = int(counts.sum())
    for sources, with_moments in ((sc.sources, True), (sc.sources, False), (bundled.sources, True),
                                  (bundled.sources, False), (sc.sources, True)):
        outs = []
        for s in (ref, gr):
            s.set_sources(sources)
            img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
            rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda") if with_moments else None
            s.trace(img, rec, mom)
            torch.cuda.synchronize()
            outs.append((img.cpu().numpy(), P.records_to_numpy(rec), None if mom is None else mom.cpu().numpy()))
        assert np.array_equal(outs[0][0], outs[1][0])
        assert np.array_equal(outs[0][1], outs[1][1])
        if with_moments:
            np.testing.assert_allclose(outs[1][2], outs[0][2], rtol=1e-12, atol=1e-15)
            assert outs[1][2][:, 0].sum() == int((outs[1][1]["flags"] & 1).sum())
    ref.close()
    gr.close()


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_sensor_extensions(oracle_mod, precision):
    """Dead layer, back-side reflection and a depth-dependent diffusion sigma from the field model."""
    counts = [6000, 3000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=12))
    sc.detector.dead_layer = 0.0003
    sc.detector.t_si = 0.01
    sc.detector.sigma = I.diffusion_sigma_table(t_si_mm=0.01, v_over=5.0, n_bulk=5e11)
    sc.back_reflect = True
    gpu = G.run_gpu(sc, precision, early_reject=True)
    ora = G.oracle_trace(oracle_mod, sc)
    reasons = (ora["flags"] >> 8) & 0xFF
    assert (reasons == 8).sum() > 50
    if precision == P.PLAIN_FP64:
        det_g, det_o = (gpu["rec"]["flags"] & 1) == 1, (ora["flags"] & 1) == 1
        assert np.all((det_g == det_o) | G.boundary_mask(ora))
        both = det_g & det_o
        err = np.maximum(np.abs(gpu["rec"]["x"][both] - ora["x"][both]), np.abs(gpu["rec"]["y"][both] - ora["y"][both]))
        assert err.max() / sc.detector.pixel < 1e-6
    G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-6 if precision == P.PLAIN_FP64 else 1e-3)


def test_bleeding_matches_oracle(oracle_mod):
    rng = np.random.default_rng(4)
    img = rng.integers(0, 300, size=(64, 96)).astype(np.uint32)
    for _ in range(12):
        img[rng.integers(0, 64), rng.integers(0, 96)] += np.uint32(rng.integers(1000, 200000))
    img[10, :] = 700
    t = torch.as_tensor(img.view(np.int32).copy(), device="cuda")
    removed = P.bleed(t, 1000)
    torch.cuda.synchronize()
    ref, ref_removed = oracle_mod.bleed(img, 1000)
    assert np.array_equal(t.cpu().numpy().view(np.uint32), ref)
    assert int(removed.item()) == ref_removed


def test_invalid_sources_are_rejected():
    sc = I.paraboloid_scene(n_photons=10)
    s = P.Scene(sc)
    bad = sc.sources.subset([0])
    bad.sed = np.array([5], np.int32)            # no such SED
    s.set_sources(bad)
    img = torch.zeros((256, 256), dtype=torch.int32, device="cuda")
    with pytest.raises(P.PhosimError) as e:
        s.trace(img)
    assert e.value.code == -1
    s.close()


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_background_bundles(oracle_mod, precision):
    """Sec. 3.2 background optimisation: a sky-like Gaussian source traced as bundles of 8 photons per ray
    (ragged ranges included) against the oracle: in FP64 photon by photon, in the mixed precisions through the
    moments; a bundle of one is the unbundled source."""
    counts = [4003, 700, 2500]
    src = G.mixed_sources(counts, seed=14)
    src.kind = np.array([I.GAUSS, I.POINT, I.GAUSS], np.int32)
    src.a = np.array([6e-5, 0.0, 3e-5])
    src.bundle = np.array([8, 1, 3], np.int32)
    src.bundle_sigma = np.array([0.003, 0.0, 0.01])
    sc = G.test_system_scene(sources=src)
    first = np.array([5, 0, 1], np.uint64)
    # photon fates are compared in full, so no dynamic transmission test (it renames some losses) in FP64
    gpu = G.run_gpu(sc, precision, early_reject=precision != P.PLAIN_FP64, first=first)
    ora = G.oracle_trace(oracle_mod, sc, first=first)
    if precision == P.PLAIN_FP64:
        r = G.compare_records(sc, gpu, ora)
        assert r["max_err_px"] < 1e-6, r
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-6)
    else:
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-3)
    assert np.array_equal(gpu["image"], G.image_from_pix(gpu["rec"], sc.detector))
    # one photon per ray: exactly the unbundled trace
    sc.sources.bundle = np.array([1, 1, 1], np.int32)
    one = G.run_gpu(sc, precision, early_reject=True, first=first)
    sc.sources.bundle = None
    sc.sources.bundle_sigma = None
    none = G.run_gpu(sc, precision, early_reject=True, first=first)
    assert np.array_equal(one["rec"], none["rec"])


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_ghosts_of_a_coated_plate_match_oracle(oracle_mod, precision):
    """Ghosts (Sec. 2.4.2) through the C ABI: the tilted beam behind a coated plate (T = 0.5, R = 0.45 on both
    faces), photon by photon against the oracle; no single-precision step is on this path except the
    wavelength blur, so every precision meets the FP64 gate."""
    from tests.test_oracle_pins import _ghost_plate_scene
    sc = _ghost_plate_scene(0.5, 0.45, n_photons=20000)
    gpu = G.run_gpu(sc, precision)
    ora = G.oracle_trace(oracle_mod, sc)
    r = G.compare_records(sc, gpu, ora)
    assert r["max_err_px"] < (1e-6 if precision == P.PLAIN_FP64 else 1e-4), r
    assert r["n_detected"] > 6000


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_ghosts_in_the_catadioptric_system(oracle_mod, precision):
    """The full test system with both filter faces coated and reflecting (R = 0.1 in band, 0.9 out of band):
    ghosts between the filter faces reach the detector, others leave backwards past the lens and the mirror,
    through the atmosphere and the sensor; the dynamic transmission test on (only the first coated surface's
    draw is certain once coatings reflect)."""
    counts = [5000, 3000, 1000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=15))
    sc.surfaces[4].coating = 0
    c = sc.coatings[0]
    c.reflect = np.where(c.table > 0, 0.3, 0.9) * np.ones_like(c.table)
    c.reflect = np.minimum(c.reflect, 1.0 - c.table)
    gpu = G.run_gpu(sc, precision, early_reject=True)
    ora = G.oracle_trace(oracle_mod, sc)
    det_g, det_o = (gpu["rec"]["flags"] & 1) == 1, (ora["flags"] & 1) == 1
    if precision == P.PLAIN_FP64:
        assert np.all((det_g == det_o) | G.boundary_mask(ora))
        both = det_g & det_o
        err = np.maximum(np.abs(gpu["rec"]["x"][both] - ora["x"][both]), np.abs(gpu["rec"]["y"][both] - ora["y"][both]))
        assert err.max() / sc.detector.pixel < 1e-6
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-6)
    else:
        G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-3)
    assert np.array_equal(gpu["image"], G.image_from_pix(gpu["rec"], sc.detector))


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_fringing_back_side_reflection(oracle_mod, precision):
    """Fringing (Sec. 2.4.2): photons crossing a thin (3 um) chip are reflected at its back with the
    single-layer interference probability at their wavelength, angle and the local optical thickness of a
    wedged layer.  FP64: fates identical to the oracle's away from flagged decisions, positions to 1e-6 pixel;
    mixed paths: moments within the 0.1 % gate.  The effect is real: replacing it by the normal-incidence
    Fresnel reflection changes the fate of some of the same photons."""
    counts = [8000, 5000]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=14))
    sc.detector.t_si = 0.003
    sc.detector.sigma = np.array([0.001, 0.001])
    sc.back_reflect = True
    sc.fringe = True
    sc.detector.t_si_gx = 3e-4
    sc.detector.t_si_gy = -1e-4
    gpu = G.run_gpu(sc, precision, early_reject=True)
    ora = G.oracle_trace(oracle_mod, sc)
    det_g, det_o = (gpu["rec"]["flags"] & 1) == 1, (ora["flags"] & 1) == 1
    if precision == P.PLAIN_FP64:
        assert np.all((det_g == det_o) | G.boundary_mask(ora))
        both = det_g & det_o
        err = np.maximum(np.abs(gpu["rec"]["x"][both] - ora["x"][both]), np.abs(gpu["rec"]["y"][both] - ora["y"][both]))
        assert err.max() / sc.detector.pixel < 1e-6
    else:
        assert np.mean(det_g != det_o) < 2e-4
    G.compare_moments(gpu["moments"], G.oracle_moments(ora, len(counts)), rel=1e-6 if precision == P.PLAIN_FP64 else 1e-3)
    # the same photons with the normal-incidence Fresnel probability: fringing changes the fate of some
    sc.fringe = False
    ora0 = G.oracle_trace(oracle_mod, sc)
    assert np.sum(det_o != ((ora0["flags"] & 1) == 1)) > 50


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED_DS])
def test_asphere_terms_of_every_order(oracle_mod, precision):
    """Sec. 2.4.1 asphere polynomials of every order against the oracle, photon by photon, without the
    atmosphere and the sensor: the paraboloid carries all four even terms alpha_4..alpha_10 (each about 10 um
    of sag at the rim; the double-single path takes its Newton root after one step there, with the slopes
    carried by the single-precision second derivatives of all four terms), and the lens's first face all four
    odd terms alpha_3..alpha_9 (about 1 um each) beside alpha_4, which the double-single path iterates to a step
    below 1e-8 mm.  Fates as the oracle's away from boundaries and positions at the FP64 per-photon gate."""
    import dataclasses
    sc = G.test_system_scene(n_photons=20000, sensor=False, atmosphere=False)
    s0, s1 = sc.surfaces[0], sc.surfaces[1]
    r0, r1 = s0.r_out, s1.r_out
    even = (1e-2 / r0 ** 4, -1e-2 / r0 ** 6, 1e-2 / r0 ** 8, -1e-2 / r0 ** 10)
    odd = (1e-3 / r1 ** 3, -1e-3 / r1 ** 5, 1e-3 / r1 ** 7, -1e-3 / r1 ** 9)
    surfaces = list(sc.surfaces)
    surfaces[0] = dataclasses.replace(s0, alpha=(0.0, even[0], 0.0, even[1], 0.0, even[2], 0.0, even[3]))
    surfaces[1] = dataclasses.replace(s1, alpha=(odd[0], s1.alpha[1], odd[1], 0.0, odd[2], 0.0, odd[3], 0.0))
    sc = dataclasses.replace(sc, surfaces=surfaces)
    gpu = G.run_gpu(sc, precision)
    ora = G.oracle_trace(oracle_mod, sc)
    r = G.compare_records(sc, gpu, ora)
    assert r["n_detected"] > 5000, r
    assert r["max_err_px"] < (1e-6 if precision == P.PLAIN_FP64 else 1e-4), r
