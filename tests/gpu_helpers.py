"""Helpers of the GPU tests: run the CUDA path through the C ABI and compare it with the oracle."""
import numpy as np

from paper_1504_06570_gb300 import inputs as I
from paper_1504_06570_gb300 import phosim as P

# photons whose path passes within these margins of an accept decision may legitimately differ
MARGIN_MM = 1e-7          # 1e-5 pixel of 10 um
MARGIN_NM = 1e-6


def run_gpu(scene, precision=P.PLAIN_FP64, records=True, moments=True, schedule=None, n_photons=None, first=None,
            host_image=False, early_reject=False, graph=False):
    import torch
    s = P.Scene(scene, precision, early_reject=early_reject, graph=graph)
    if schedule:
        s.set_schedule(*schedule)
    cnt = scene.sources.n_photons if n_photons is None else np.asarray(n_photons, np.uint64)
    n = int(np.sum(cnt))
    d = scene.detector
    dev = "cpu" if host_image else "cuda"
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
    rec = torch.zeros(max(1, n) * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda") if records else None
    mom = torch.zeros((len(scene.sources), P.MOMENT_WORDS), dtype=torch.float64, device="cuda") if moments else None
    s.trace(img, rec, mom, n_photons=cnt, first=first)
    torch.cuda.synchronize()
    out = {"image": img.cpu().numpy().view(np.uint32), "counters": s.counters()}
    if records:
        out["rec"] = P.records_to_numpy(rec)[:n]
    if moments:
        out["moments"] = mom.cpu().numpy()
    s.close()
    return out


def oracle_trace(oracle_mod, scene, n_photons=None, first=None):
    o = oracle_mod.Oracle(scene)
    return o.trace(count=n_photons, first=first, n_threads=8)


def boundary_mask(ora):
    return (ora["margin_mm"] < MARGIN_MM) | (ora["margin_nm"] < MARGIN_NM)


def compare_records(scene, gpu, ora, pos_tol_px=1e-4, min_frac=0.99999):
    """Per-photon parity: identical accept decisions except at flagged boundaries, final positions within
    pos_tol_px pixels for at least min_frac of the photons detected by both, identical pixels."""
    rec = gpu["rec"]
    bnd = boundary_mask(ora)
    same = rec["flags"] == ora["flags"]
    assert np.all(same | bnd), f"{np.sum(~same & ~bnd)} photons differ in their fate away from any boundary"
    both = ((rec["flags"] & 1) == 1) & ((ora["flags"] & 1) == 1)
    px = scene.detector.pixel
    err = np.maximum(np.abs(rec["x"][both] - ora["x"][both]), np.abs(rec["y"][both] - ora["y"][both])) / px
    frac = np.mean(err <= pos_tol_px) if len(err) else 1.0
    assert frac >= min_frac, (frac, np.max(err))
    okpix = both & ~bnd
    assert np.array_equal(rec["pix"][okpix], ora["pix"][okpix])
    lam_err = np.max(np.abs(rec["lam"] - ora["lam"])) if len(rec) else 0.0
    return {"max_err_px": float(np.max(err)) if len(err) else 0.0, "frac": float(frac), "lam_err": float(lam_err),
            "n_boundary": int(np.sum(bnd)), "n_detected": int(np.sum(both))}


def image_from_pix(rec, det):
    m = (rec["flags"] & 1) == 1
    return np.bincount(rec["pix"][m], minlength=det.nx * det.ny).reshape(det.ny, det.nx).astype(np.uint32)


def oracle_moments(ora, n_src):
    out = np.zeros((n_src, 6))
    det = (ora["flags"] & 1) == 1
    for s in range(n_src):
        m = det & (ora["source"] == s)
        x, y = ora["x"][m], ora["y"][m]
        if len(x):
            mx, my = x.mean(), y.mean()
            out[s] = [len(x), mx, my, ((x - mx) ** 2).mean(), ((x - mx) * (y - my)).mean(), ((y - my) ** 2).mean()]
    return out


def compare_moments(gpu_m, ora_m, rel=1e-3):
    """Centroids within rel * PSF size, second moments within rel (relative), counts exact or within the
    boundary photons."""
    g = P.derived_moments(gpu_m)
    for s in range(len(ora_m)):
        if ora_m[s, 0] < 10:
            continue
        size = np.sqrt(ora_m[s, 3] + ora_m[s, 5])
        assert abs(g[s, 1] - ora_m[s, 1]) <= rel * size, (s, g[s], ora_m[s])
        assert abs(g[s, 2] - ora_m[s, 2]) <= rel * size, (s, g[s], ora_m[s])
        T = ora_m[s, 3] + ora_m[s, 5]
        for k in (3, 4, 5):
            assert abs(g[s, k] - ora_m[s, k]) <= rel * T, (s, k, g[s], ora_m[s])
    return g


_HF = None


def hf_table():
    global _HF
    if _HF is None:
        _HF = I.high_frequency_kick_table(K=1024)[0]
    return _HF


def test_system_scene(n_photons=40000, sensor=True, atmosphere=True, chip=512, sources=None, screen_n=256, hf=False):
    """A small catadioptric system exercising every surface feature: an annular paraboloid with a
    Zernike figure and a tilt, a decentred aspheric meniscus lens, a coated filter plate, a detector."""
    mats = [I.Material(I.VACUUM), I.Material(I.SELLMEIER, I.FUSED_SILICA_B, I.FUSED_SILICA_C), I.Material(I.SILICON)]
    coat = I.filter_coating(450.0, 650.0, 0.9, lam0=400.0, nlam=300)
    zern = [0.0, 0.0, 0.0, 3e-5, 2e-5, -1e-5, 1e-5, 0.0, 0.0, 0.0, 5e-6]
    surfaces = [
        I.Surface(kind=I.MIRROR, R=20000.0, kappa=-1.0, z=0.0, r_in=100.0, r_out=500.0, zern_rnorm=500.0, zern=zern,
                  pert=(0.0, 0.0, 0.0, 2e-6, -1e-6, 0.0)),
        I.Surface(kind=I.REFRACT, R=5000.0, kappa=-0.5, alpha=(0, 2e-12, 0, 0, 0, 0, 0, 0), z=9500.0, r_out=60.0,
                  material=1, pert=(0.05, -0.02, 0.0, 0.0, 0.0, 0.0)),
        I.Surface(kind=I.REFRACT, R=5200.0, z=9520.0, r_out=60.0, material=0, pert=(0.05, -0.02, 0.0, 0.0, 0.0, 0.0)),
        I.Surface(kind=I.REFRACT, R=0.0, z=9700.0, r_out=40.0, material=1, coating=0),
        I.Surface(kind=I.REFRACT, R=0.0, z=9705.0, r_out=40.0, material=0),
        I.Surface(kind=I.DETECTOR, R=0.0, z=10007.5, material=2),
    ]
    nb = 300
    det = I.Detector(nx=chip, ny=chip, pixel=0.01, t_si=0.1, ell_lam0=400.0, ell_dlam=1.0,
                     ell=I.absorption_length_table(400.0, 1.0, nb + 1), sigma=np.array([0.002, 0.003, 0.004]))
    layers = []
    if atmosphere:
        rng = np.random.default_rng(21)
        ph = I.phase_screen(screen_n, 0.04, 0.15, 20.0, rng)
        ph2 = I.phase_screen(64, 2.56, 0.15, 20.0, rng, keep="low", fcut=1.0 / (2 * screen_n * 0.04))
        layers = [I.Layer(z=8.0e6, vx=3000.0, vy=-5000.0, scales=[I.ScreenScale(40.0, ph), I.ScreenScale(2560.0, ph2)]),
                  I.Layer(z=2.0e6, vx=-1000.0, vy=2000.0, scales=[I.ScreenScale(40.0, np.roll(ph, 77, 0) * 0.7)])]
    if sources is None:
        sources = I.point_sources([0.0], [0.0], [n_photons])
    return I.Scene(seed=12345, pupil_r_in=100.0, pupil_r_out=500.0, surfaces=surfaces, materials=mats, coatings=[coat],
                   detector=det, layers=layers, sed_lam0=400.0, sed_dlam=1.0, sed_flux=I.sed_tables([5800.0, 3500.0], 400.0, 1.0, nb),
                   sersic=np.stack([I.sersic_radius_table(1.0, 256), I.sersic_radius_table(3.5, 256)]), sources=sources,
                   atmosphere=atmosphere, sensor=sensor, hf_kick=hf_table() if hf else None)


def mixed_sources(counts, seed=3):
    """Point, Sersic and Gaussian sources at small field angles (test system scale: 2e-5 rad ~ 20 px)."""
    rng = np.random.default_rng(seed)
    n = len(counts)
    kind = np.array([(I.POINT, I.SERSIC, I.GAUSS)[i % 3] for i in range(n)], np.int32)
    return I.Sources(kind=kind, sed=(np.arange(n) % 2).astype(np.int32), xi=rng.uniform(-8e-5, 8e-5, n),
                     eta=rng.uniform(-8e-5, 8e-5, n), redshift=np.where(np.arange(n) % 4 == 1, 0.1, 0.0),
                     t0=rng.uniform(0, 5, n), t_exp=np.full(n, 15.0), a=np.full(n, 3e-6), b=np.full(n, 1.5e-6),
                     pa=rng.uniform(0, np.pi, n), table=(np.arange(n) % 2).astype(np.int32),
                     n_photons=np.asarray(counts, np.uint64))
