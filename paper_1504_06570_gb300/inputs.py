"""Seeded synthetic scenes for the photon Monte Carlo path.

This module describes WHAT is simulated: optical prescriptions, phase screens, spectra, sensor tables and
source catalogues, all generated from recorded seeds.  Both the CUDA path and the CPU oracle consume the
same scene objects; neither side's per-photon arithmetic lives here.  What the paper computes before the
photon loop starts (screen synthesis, Sec. 2.3.1; the blackbody SED, Sec. 2.2; the Rajkanan absorption
coefficient, Sec. 2.4.2; the Sersic radial distribution, Sec. 2.2.1) is produced here as tables, because
the photon path itself only looks those tables up.

Units: lengths in mm, angles in rad, wavelengths in nm, times in s, phases in rad at LAMBDA_REF_NM.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

LAMBDA_REF_NM = 500.0
H_TOP_MM = 100.0e6           # top of the atmosphere, 100 km (Sec. 2.2)

# surface kinds
MIRROR, REFRACT, DETECTOR = 0, 1, 2
# material kinds
VACUUM, SELLMEIER, SILICON = 0, 1, 2
# source kinds
POINT, SERSIC, GAUSS = 0, 1, 2

# fused silica Sellmeier coefficients of Malitson (1965), lambda in um, C in um^2
FUSED_SILICA_B = (0.6961663, 0.4079426, 0.8974794)
FUSED_SILICA_C = (0.0684043 ** 2, 0.1162414 ** 2, 9.896161 ** 2)

ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0


@dataclass
class Material:
    kind: int = VACUUM
    B: Sequence[float] = (0.0, 0.0, 0.0)
    C: Sequence[float] = (0.0, 0.0, 0.0)


@dataclass
class Coating:
    """Transmission probability T(lambda, theta), and optionally reflection probability R, piecewise constant on
    a uniform grid (the paper's angle/wavelength coating interface, Sec. 2.4.2)."""
    lam0: float
    dlam: float
    theta0: float
    dtheta: float
    table: np.ndarray            # shape (n_lambda, n_theta), float64 in [0, 1]
    reflect: np.ndarray = None   # reflection probability R on the same grid (ghosts, Sec. 2.4.2); T + R <= 1


@dataclass
class Surface:
    kind: int
    R: float = 0.0               # radius of curvature (mm); 0 = flat
    kappa: float = 0.0
    alpha: Sequence[float] = (0.0,) * 8      # alpha_3 .. alpha_10, units mm^(1-i)
    z: float = 0.0               # vertex position on the optical axis (mm)
    r_in: float = 0.0            # clear aperture (mm), photons outside are removed
    r_out: float = 1.0e30
    material: int = 0            # medium after a refracting surface (index into Scene.materials)
    coating: int = -1            # index into Scene.coatings, -1 = none
    pert: Sequence[float] = (0.0,) * 6       # dx, dy, dz (mm), tx, ty, tz (rad)
    zern_rnorm: float = 0.0      # normalisation radius of the Zernike figure (mm)
    zern: Sequence[float] = ()   # Noll coefficients c_1..c_J (mm of sag)


@dataclass
class Detector:
    nx: int
    ny: int
    pixel: float                 # mm
    x0: float = 0.0              # chip centre in the detector surface frame (mm)
    y0: float = 0.0
    t_si: float = 0.1            # silicon thickness (mm)
    ell_lam0: float = 300.0      # absorption length table: lambda grid (nm) and values (mm)
    ell_dlam: float = 1.0
    ell: np.ndarray = None
    sigma: np.ndarray = None     # diffusion sigma (mm) at depths uniformly spaced over [0, t_si]
    dead_layer: float = 0.0      # field-free layer at the entrance (mm)
    t_si_gx: float = 0.0         # gradient of the silicon's optical thickness across the chip (mm per mm), for
    t_si_gy: float = 0.0         # the fringing calculation: t_si + t_si_gx (x - x0) + t_si_gy (y - y0)


@dataclass
class ScreenScale:
    pixel: float                 # mm
    phase: np.ndarray            # (N, N) float64, rad at LAMBDA_REF_NM, row = y index, column = x index


@dataclass
class Layer:
    z: float                     # altitude of the layer in the telescope frame (mm)
    vx: float = 0.0              # wind (mm/s)
    vy: float = 0.0
    scales: List[ScreenScale] = field(default_factory=list)


@dataclass
class Sources:
    kind: np.ndarray             # int32
    sed: np.ndarray              # int32, index into the SED tables
    xi: np.ndarray               # tangent-plane direction components (rad), Sec. 2.2
    eta: np.ndarray
    redshift: np.ndarray
    t0: np.ndarray
    t_exp: np.ndarray
    a: np.ndarray                # Sersic semi-major axis at r = r_e (rad); Gaussian sigma (rad)
    b: np.ndarray                # Sersic semi-minor axis (rad)
    pa: np.ndarray               # position angle (rad)
    table: np.ndarray            # int32, Sersic radial table index
    n_photons: np.ndarray        # uint64
    bundle: np.ndarray = None    # int32, photons per ray (Sec. 3.2 background optimisation); None or <= 1: one
    bundle_sigma: np.ndarray = None   # float64, sigma (mm) of the spread of a ray's photons on the detector

    def __len__(self):
        return len(self.kind)

    def subset(self, idx):
        return Sources(**{f.name: (None if getattr(self, f.name) is None else np.asarray(getattr(self, f.name))[idx])
                          for f in dataclasses.fields(self)})


@dataclass
class Scene:
    seed: int
    pupil_r_in: float
    pupil_r_out: float
    surfaces: List[Surface]
    materials: List[Material]
    coatings: List[Coating]
    detector: Detector
    layers: List[Layer]
    sed_lam0: float
    sed_dlam: float
    sed_flux: np.ndarray         # (n_sed, n_bins) flux density per unit wavelength
    sersic: np.ndarray           # (n_tables, K) radius in units of r_e at u = (k + 0.5) / K
    sources: Sources
    h_top: float = H_TOP_MM
    lambda_ref: float = LAMBDA_REF_NM
    atmosphere: bool = True
    sensor: bool = True          # False: record the hit on the detector surface, no silicon
    z_entrance: float = None     # plane (mm) where the raytrace starts, below every layer, above every optic
    hf_kick: np.ndarray = None   # quantiles (rad at lambda_ref) of the high-frequency kick, or None
    back_reflect: bool = False   # back-side reflection of photons that cross the silicon
    fringe: bool = False         # with back_reflect: the reflection probability from the single-layer
                                 # interference calculation (fringing) instead of the normal-incidence Fresnel one

    def __post_init__(self):
        if self.z_entrance is None:
            self.z_entrance = max(s.z for s in self.surfaces) + 1000.0


# ----------------------------------------------------------------------------------------------------------
# tables the paper computes before the photon loop
# ----------------------------------------------------------------------------------------------------------

def blackbody_flux(T_K, lam_nm):
    """Planck spectral radiance per unit wavelength (arbitrary overall scale) at lam_nm."""
    h, c, k = 6.62607015e-34, 2.99792458e8, 1.380649e-23
    lam = np.asarray(lam_nm, dtype=np.float64) * 1e-9
    x = h * c / (lam * k * np.asarray(T_K, dtype=np.float64)[..., None])
    return (1.0 / lam ** 5) / np.expm1(x) * 1e-30


def sed_tables(temps_K, lam0=300.0, dlam=1.0, nbins=900):
    centres = lam0 + (np.arange(nbins) + 0.5) * dlam
    return blackbody_flux(np.atleast_1d(temps_K), centres)


def rajkanan_alpha_per_cm(lam_nm, T_K=173.0):
    """Absorption coefficient of silicon (1/cm) from the Rajkanan model with the constants of Sec. 2.4.2.
    Each squared term contributes only where its base is positive; the direct-gap term only above E_gd."""
    E = 1239.841984 / np.asarray(lam_nm, dtype=np.float64)
    kT = 8.617333262e-5 * T_K
    beta, gamma = 7.021e-4, 1108.0
    shift = beta * T_K * T_K / (T_K + gamma)
    Eg = (1.1557 - shift, 2.5 - shift)
    Egd = 3.2 - shift
    Ep = (1.827e-2, 5.773e-2)
    C = (5.5, 4.0)
    A = (3.231e2, 7.237e3)
    Ad = 1.052e6
    alpha = np.zeros_like(E)
    for i in range(2):
        for j in range(2):
            b1 = E - Eg[j] + Ep[i]
            b2 = E - Eg[j] - Ep[i]
            t1 = np.where(b1 > 0, b1 * b1, 0.0) / np.expm1(Ep[i] / kT)
            t2 = np.where(b2 > 0, b2 * b2, 0.0) / (-np.expm1(-Ep[i] / kT))
            alpha += C[i] * A[j] * (t1 + t2)
    alpha += Ad * np.sqrt(np.clip(E - Egd, 0.0, None))
    return alpha


def absorption_length_table(lam0=300.0, dlam=1.0, n=901, T_K=173.0):
    lam = lam0 + np.arange(n) * dlam
    alpha = rajkanan_alpha_per_cm(lam, T_K)
    return 10.0 / np.maximum(alpha, 1e-5)              # mm; below the band gap: 1 km, i.e. never converts


def sersic_bn(n):
    from scipy.special import gammaincinv
    return float(gammaincinv(2.0 * n, 0.5))


def sersic_radius_table(n, K=1024):
    """Inverse cumulative distribution of the radius (units of the half-light radius) of a circular
    Sersic profile I(r) ~ exp(-b_n r^(1/n)) (Sec. 2.2.1), sampled at u = (k + 0.5) / K."""
    from scipy.special import gammaincinv
    bn = sersic_bn(n)
    u = (np.arange(K) + 0.5) / K
    return (gammaincinv(2.0 * n, u) / bn) ** n


# ----------------------------------------------------------------------------------------------------------
# phase screens (Sec. 2.3.1): FFT synthesis with subharmonics
# ----------------------------------------------------------------------------------------------------------

PSD_CONST = 0.023   # phase PSD 0.023 r0^(-5/3) f^(-11/3), f in cycles per metre


def phase_psd(f2, r0_m, L0_m):
    inv_L0_2 = 0.0 if not np.isfinite(L0_m) else 1.0 / (L0_m * L0_m)
    with np.errstate(divide="ignore"):
        return PSD_CONST * r0_m ** (-5.0 / 3.0) * (f2 + inv_L0_2) ** (-11.0 / 6.0)


def _cell_power(fx, fy, dfc, r0_m, L0_m, nq=8):
    """Power of the PSD integrated over the square cell of side dfc centred on (fx, fy) (Gauss-Legendre),
    given to the single mode that stands for the cell.  Near the origin the PSD changes by orders of
    magnitude across a cell, so its midpoint value under-represents the cell's variance."""
    x, w = np.polynomial.legendre.leggauss(nq)
    x = 0.5 * x * dfc
    w = 0.5 * w
    FX = np.asarray(fx)[..., None, None] + x[:, None]
    FY = np.asarray(fy)[..., None, None] + x[None, :]
    return (phase_psd(FX * FX + FY * FY, r0_m, L0_m) * (w[:, None] * w[None, :])).sum((-1, -2)) * dfc * dfc


def fft_mode_power(N, pix_m, r0_m, L0_m, keep="all", fcut=None):
    """Variance given to each FFT mode of an N x N screen (layout of numpy.fft.fftfreq)."""
    df = 1.0 / (N * pix_m)
    f = np.fft.fftfreq(N, pix_m)
    fx, fy = np.meshgrid(f, f)
    power = phase_psd(fx * fx + fy * fy, r0_m, L0_m) * df * df
    power[0, 0] = 0.0
    if keep == "low":
        return np.where((np.abs(fx) < fcut) & (np.abs(fy) < fcut), power, 0.0)
    m = np.fft.fftfreq(N, 1.0 / N).astype(int)
    near = np.where(np.abs(m) <= 3)[0]
    for iy in near:
        for ix in near:
            if iy or ix:
                power[iy, ix] = _cell_power(fx[iy, ix], fy[iy, ix], df, r0_m, L0_m)
    return power


def phase_screen(N, pix_m, r0_m, L0_m, rng, subharmonics=0, keep="all", fcut=None):
    """Periodic N x N screen of phase (rad at 500 nm) with pixel pix_m metres (FFT synthesis).

    keep="all": every FFT mode except f = 0 (cells next to the origin carry their cell-integrated power),
    plus `subharmonics` levels of 3 x 3 sub-harmonic cells that represent the origin's cell (they make the
    screen non-periodic).  keep="low": only modes with |fx| < fcut and |fy| < fcut (the coarse scale of a
    two-scale pair), each with its midpoint power.
    """
    df = 1.0 / (N * pix_m)
    power = fft_mode_power(N, pix_m, r0_m, L0_m, keep, fcut)
    cn = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * np.sqrt(power)
    phs = np.fft.ifft2(cn).real * (N * N)
    if keep == "all" and subharmonics:
        x = np.arange(N) * pix_m
        X, Y = np.meshgrid(x, x)
        lo = np.zeros((N, N))
        for p in range(1, subharmonics + 1):
            dfp = df / 3.0 ** p
            for m in (-1, 0, 1):
                for n in (-1, 0, 1):
                    if m == 0 and n == 0:
                        continue
                    fxp, fyp = m * dfp, n * dfp
                    amp = np.sqrt(_cell_power(fxp, fyp, dfp, r0_m, L0_m))
                    c = (rng.standard_normal() + 1j * rng.standard_normal()) * amp
                    lo += (c * np.exp(2j * np.pi * (fxp * X + fyp * Y))).real
        phs = phs + lo - lo.mean()
    return phs


# ----------------------------------------------------------------------------------------------------------
# sources
# ----------------------------------------------------------------------------------------------------------

def point_sources(xi, eta, n_photons, sed=None, t0=0.0, t_exp=15.0):
    n = len(xi)
    z = np.zeros(n)
    return Sources(kind=np.full(n, POINT, np.int32),
                   sed=np.zeros(n, np.int32) if sed is None else np.asarray(sed, np.int32),
                   xi=np.asarray(xi, np.float64), eta=np.asarray(eta, np.float64), redshift=z.copy(),
                   t0=np.full(n, t0), t_exp=np.full(n, t_exp), a=z.copy(), b=z.copy(), pa=z.copy(),
                   table=np.zeros(n, np.int32), n_photons=np.asarray(n_photons, np.uint64))


def concat_sources(parts: Sequence[Sources]) -> Sources:
    defaults = {"bundle": (np.int32, 1), "bundle_sigma": (np.float64, 0.0)}

    def field(p, name):
        v = getattr(p, name)
        if v is None:
            dt, fill = defaults[name]
            return np.full(len(p), fill, dt)
        return np.asarray(v)
    out = {}
    for f in dataclasses.fields(Sources):
        if f.name in defaults and all(getattr(p, f.name) is None for p in parts):
            out[f.name] = None
        else:
            out[f.name] = np.concatenate([field(p, f.name) for p in parts])
    return Sources(**out)


# ----------------------------------------------------------------------------------------------------------
# scene recipes
# ----------------------------------------------------------------------------------------------------------

def _sensor(nx, pixel, lam0, nlam, t_si=0.1, sigma=0.003):
    return Detector(nx=nx, ny=nx, pixel=pixel, t_si=t_si, ell_lam0=lam0, ell_dlam=1.0,
                    ell=absorption_length_table(lam0, 1.0, nlam + 1), sigma=np.array([sigma, sigma]))


def paraboloid_scene(n_photons=100_000, seed=1, screen_n=512, screen_pix_mm=20.0, r0_m=0.15,
                     layer_z_mm=5.0e6, atmosphere=True, sensor=True, screen_seed=11, xi=0.0, eta=0.0,
                     sed_T=5800.0, lam_lo=400.0, lam_hi=700.0, chip=256):
    """One on-axis star through one frozen Kolmogorov screen onto a D = 1 m f/10 paraboloid and a
    chip of 10 um pixels behind 100 um of silicon (the plain-method tiny case)."""
    R = 20000.0
    surfaces = [Surface(kind=MIRROR, R=R, kappa=-1.0, z=0.0, r_in=0.0, r_out=500.0),
                Surface(kind=DETECTOR, R=0.0, z=R / 2.0, material=1)]
    materials = [Material(VACUUM), Material(SILICON)]
    nb = int(round(lam_hi - lam_lo))
    layers = []
    if atmosphere:
        # sub-harmonics restore the low-frequency power the FFT lattice misses; they make the screen
        # non-periodic, so it is rolled by half a screen to put the seam 5 m away from the pupil (v = 0)
        rng = np.random.default_rng(screen_seed)
        ph = phase_screen(screen_n, screen_pix_mm * 1e-3, r0_m, np.inf, rng, subharmonics=3)
        ph = np.roll(ph, (screen_n // 2, screen_n // 2), (0, 1))
        layers = [Layer(z=layer_z_mm, scales=[ScreenScale(screen_pix_mm, ph)])]
    src = point_sources([xi], [eta], [n_photons])
    return Scene(seed=seed, pupil_r_in=0.0, pupil_r_out=500.0, surfaces=surfaces, materials=materials,
                 coatings=[], detector=_sensor(chip, 0.01, lam_lo, nb), layers=layers, sed_lam0=lam_lo,
                 sed_dlam=1.0, sed_flux=sed_tables([sed_T], lam_lo, 1.0, nb), sersic=np.ones((1, 4)),
                 sources=src, atmosphere=atmosphere, sensor=sensor)


def cn2_weights(rng, n_layers=7):
    """Relative turbulence integral per layer: one log-normal draw for the ground layer and one shared by
    the free-atmosphere layers (Sec. 2.3.1), applied to a fixed base profile and normalised to 1."""
    base = np.array([0.45, 0.10, 0.10, 0.10, 0.10, 0.08, 0.07])[:n_layers]
    g_ground, g_free = rng.standard_normal(2)
    w = base * np.exp(0.4 * np.r_[g_ground, np.full(n_layers - 1, g_free)])
    return w / w.sum()


LAYER_HEIGHTS_KM = (0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0)
ATM_Z0_MM = 25_000.0     # telescope-frame height of altitude 0: above every optical surface


def von_karman_layers(seed=7, r0_m=0.15, L0_m=20.0, fine_n=4096, fine_pix_mm=10.0, coarse_n=1024,
                      coarse_pix_mm=640.0, heights_km=LAYER_HEIGHTS_KM, wind_scale_m_s=10.0):
    """Seven frozen-flow layers, each a fine screen plus a coarse screen holding the modes too long for
    the fine one (two of the paper's pixel scales, Sec. 2.3.1)."""
    rng = np.random.default_rng(seed)
    w = cn2_weights(rng, len(heights_km))
    fcut = 1.0 / (2.0 * fine_n * fine_pix_mm * 1e-3)
    layers = []
    for k, h in enumerate(heights_km):
        r0k = r0_m * w[k] ** (-3.0 / 5.0)
        fine = phase_screen(fine_n, fine_pix_mm * 1e-3, r0k, L0_m, rng, subharmonics=0)
        coarse = phase_screen(coarse_n, coarse_pix_mm * 1e-3, r0k, L0_m, rng, subharmonics=0, keep="low",
                              fcut=fcut)
        speed = wind_scale_m_s * math.sqrt(-math.log(1.0 - rng.random()))    # Weibull, k = 2
        ang = 2.0 * math.pi * rng.random()
        layers.append(Layer(z=ATM_Z0_MM + h * 1e6, vx=speed * 1e3 * math.cos(ang), vy=speed * 1e3 * math.sin(ang),
                            scales=[ScreenScale(fine_pix_mm, fine), ScreenScale(coarse_pix_mm, coarse)]))
    layers.sort(key=lambda L: -L.z)
    return layers


DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


def load_optics_json(path):
    with open(path) as f:
        d = json.load(f)
    surfaces = [Surface(**s) for s in d["surfaces"]]
    materials = [Material(**m) for m in d["materials"]]
    return d, surfaces, materials


def filter_coating(lo=550.0, hi=700.0, T_in=0.95, lam0=300.0, nlam=900):
    lam = lam0 + np.arange(nlam) + 0.5
    T = np.where((lam > lo) & (lam < hi), T_in, 0.0)
    return Coating(lam0=lam0, dlam=1.0, theta0=0.0, dtheta=math.pi / 2, table=T[:, None].copy())


# ----------------------------------------------------------------------------------------------------------
# the large workload: synthetic three-mirror survey telescope, seven-layer atmosphere, 1000 stars
# ----------------------------------------------------------------------------------------------------------

THREE_MIRROR_JSON = os.path.join(DATA_DIR, "three_mirror_camera.json")


def three_mirror_optics():
    """Surfaces and media of the synthetic 8.4 m three-mirror telescope and three-lens camera (f/1.23,
    plate scale ~20 arcsec/mm), with the 550-700 nm top-hat filter coating on the filter's first face."""
    d, surfaces, materials = load_optics_json(THREE_MIRROR_JSON)
    return d, surfaces, materials


def star_field(n_stars, n_total, rng, half_field_deg=0.1, m_lo=16.0, m_hi=22.0, t_exp=15.0):
    """Stars uniform over a square field, magnitudes from N(<m) ~ 10^(0.3 m) on [m_lo, m_hi], photon
    counts ~ 10^(-0.4 m) normalised to n_total, one blackbody SED per star (T uniform 3000-10000 K)."""
    h = math.radians(half_field_deg)
    xi, eta = rng.uniform(-h, h, n_stars), rng.uniform(-h, h, n_stars)
    a, b = 10 ** (0.3 * m_lo), 10 ** (0.3 * m_hi)
    m = np.log10(a + rng.random(n_stars) * (b - a)) / 0.3
    w = 10 ** (-0.4 * m)
    counts = np.floor(w / w.sum() * n_total).astype(np.uint64)
    counts[np.argmax(counts)] += np.uint64(n_total - int(counts.sum()))
    temps = rng.uniform(3000.0, 10000.0, n_stars)
    src = point_sources(xi, eta, counts, sed=np.arange(n_stars), t_exp=t_exp)
    return src, temps, m


def three_mirror_scene(n_stars=1000, n_total=100_000_000, seed=2, atmosphere=True, sensor=True, screen_seed=7,
                       fine_n=4096, coarse_n=1024, sources=None):
    """The large workload: 1000 stars (1e8 photons, 300-1200 nm blackbodies) through seven von Karman
    layers (L0 = 20 m, 4096^2 at 1 cm plus 1024^2 at 64 cm each) and the three-mirror telescope onto one
    4096 x 4096 chip of 10 um pixels.  fine_n / coarse_n shrink the screens (pixel sizes kept) for tests."""
    d, surfaces, materials = three_mirror_optics()
    rng = np.random.default_rng(seed)
    if sources is None:
        sources, temps, _ = star_field(n_stars, n_total, rng)
    else:
        temps = rng.uniform(3000.0, 10000.0, int(np.max(sources.sed)) + 1)
    layers = von_karman_layers(seed=screen_seed, fine_n=fine_n, coarse_n=coarse_n,
                               coarse_pix_mm=640.0 * 1024 / coarse_n * (fine_n / 4096)) if atmosphere else []
    det = Detector(nx=4096, ny=4096, pixel=0.01, t_si=0.1, ell_lam0=300.0, ell_dlam=1.0,
                   ell=absorption_length_table(300.0, 1.0, 901), sigma=np.array([0.003, 0.003]))
    return Scene(seed=seed, pupil_r_in=d["pupil_r_in"], pupil_r_out=d["pupil_r_out"], surfaces=surfaces,
                 materials=materials, coatings=[filter_coating(550.0, 700.0, 0.95, lam0=300.0, nlam=900)],
                 detector=det, layers=layers, sed_lam0=300.0, sed_dlam=1.0, sed_flux=sed_tables(temps, 300.0, 1.0, 900),
                 sersic=np.ones((1, 4)), sources=sources, atmosphere=atmosphere, sensor=sensor, z_entrance=ATM_Z0_MM - 1000.0)


def galaxy_and_star_catalog(n_sources, rng, half_field_deg=0.1, star_frac=0.7, lo=1e2, hi=1e7, n_index_levels=64,
                            t_exp=15.0):
    """Stars (70 %) and Sersic galaxies (30 %): index n uniform on [0.5, 4] (snapped to 64 levels so the
    radial tables are shared), half-light radius log-uniform 0.2-3 arcsec, ellipticity |e| < 0.6 uniform in
    the disk, photon counts log-uniform on [lo, hi].  Returns (sources, SED temperatures, Sersic tables)."""
    h = math.radians(half_field_deg)
    n_star = int(round(star_frac * n_sources))
    kind = np.r_[np.full(n_star, POINT), np.full(n_sources - n_star, SERSIC)].astype(np.int32)
    rng.shuffle(kind)
    xi, eta = rng.uniform(-h, h, n_sources), rng.uniform(-h, h, n_sources)
    counts = np.exp(rng.uniform(math.log(lo), math.log(hi), n_sources)).astype(np.uint64)
    levels = 0.5 + np.arange(n_index_levels) * (3.5 / (n_index_levels - 1))
    n_idx = rng.uniform(0.5, 4.0, n_sources)
    table = np.clip(np.rint((n_idx - 0.5) / (3.5 / (n_index_levels - 1))), 0, n_index_levels - 1).astype(np.int32)
    re = np.exp(rng.uniform(math.log(0.2), math.log(3.0), n_sources)) * ARCSEC
    er, ephi = 0.6 * np.sqrt(rng.random(n_sources)), rng.uniform(0, math.pi, n_sources)
    q = (1 - er) / (1 + er)
    a, b = re / np.sqrt(q), re * np.sqrt(q)
    a = np.where(kind == SERSIC, a, 0.0)
    b = np.where(kind == SERSIC, b, 0.0)
    temps = rng.uniform(3000.0, 10000.0, n_sources)
    src = Sources(kind=kind, sed=np.arange(n_sources, dtype=np.int32), xi=xi, eta=eta, redshift=np.zeros(n_sources),
                  t0=np.zeros(n_sources), t_exp=np.full(n_sources, t_exp), a=a, b=b, pa=ephi,
                  table=np.where(kind == SERSIC, table, 0).astype(np.int32), n_photons=counts)
    tables = np.stack([sersic_radius_table(n, 1024) for n in levels])
    return src, temps, tables


def background_nodes(n_photons, chip_half_mm, plate_arcsec_per_mm, sed_index, spacing_arcsec=15.0, t_exp=15.0,
                     bundle=1, bundle_sigma_arcsec=0.0):
    """Diffuse sky as Gaussian sources (sigma = spacing) on a square grid every 15 arcsec covering the chip
    plus one spacing of margin (Sec. 2.2.2); the photons are split equally.  bundle > 1: each ray carries that
    many photons, spread on the detector with a Gaussian of bundle_sigma_arcsec (Sec. 3.2)."""
    half = chip_half_mm * plate_arcsec_per_mm + spacing_arcsec
    k = int(math.ceil(half / spacing_arcsec))
    g = np.arange(-k, k + 1) * spacing_arcsec * ARCSEC
    X, Y = np.meshgrid(g, g)
    n = X.size
    per = np.full(n, n_photons // n, np.uint64)
    per[: int(n_photons - per.sum())] += np.uint64(1)
    return Sources(kind=np.full(n, GAUSS, np.int32), sed=np.full(n, sed_index, np.int32), xi=X.ravel(), eta=Y.ravel(),
                   redshift=np.zeros(n), t0=np.zeros(n), t_exp=np.full(n, t_exp), a=np.full(n, spacing_arcsec * ARCSEC),
                   b=np.zeros(n), pa=np.zeros(n), table=np.zeros(n, np.int32), n_photons=per,
                   bundle=np.full(n, bundle, np.int32),
                   bundle_sigma=np.full(n, bundle_sigma_arcsec / plate_arcsec_per_mm))


def batched_scene(n_sources=10_000, background_photons=1_000_000_000, seed=4, fine_n=4096, coarse_n=1024,
                  photon_scale=1.0, sky_bundle=8, sky_bundle_sigma_arcsec=5.0):
    """The batched workload: 10^4 stars and galaxies (counts log-uniform 1e2-1e7, ~5e9 photons) plus 1e9
    sky-background photons on 15 arcsec nodes, through the three-mirror optics and seven-layer atmosphere.
    photon_scale multiplies every count (sub-sampled runs).  The sky uses the background optimisation of
    Sec. 3.2: rays of sky_bundle photons (about the square root of the ~60 sky photons per pixel) spread by
    sky_bundle_sigma_arcsec on the detector; sky_bundle = 1 traces every sky photon on its own."""
    d, surfaces, materials = three_mirror_optics()
    rng = np.random.default_rng(seed)
    src, temps, tables = galaxy_and_star_catalog(n_sources, rng)
    sky = background_nodes(int(background_photons), 0.5 * 4096 * 0.01, d["plate_scale_arcsec_per_mm"], n_sources,
                           bundle=sky_bundle, bundle_sigma_arcsec=sky_bundle_sigma_arcsec)
    sources = concat_sources([src, sky])
    if photon_scale != 1.0:
        sources.n_photons = np.maximum(1, np.rint(sources.n_photons * photon_scale)).astype(np.uint64)
    temps = np.r_[temps, 5800.0]
    layers = von_karman_layers(fine_n=fine_n, coarse_n=coarse_n,
                               coarse_pix_mm=640.0 * 1024 / coarse_n * (fine_n / 4096))
    det = Detector(nx=4096, ny=4096, pixel=0.01, t_si=0.1, ell_lam0=300.0, ell_dlam=1.0,
                   ell=absorption_length_table(300.0, 1.0, 901), sigma=np.array([0.003, 0.003]))
    return Scene(seed=seed, pupil_r_in=d["pupil_r_in"], pupil_r_out=d["pupil_r_out"], surfaces=surfaces,
                 materials=materials, coatings=[filter_coating(550.0, 700.0, 0.95, lam0=300.0, nlam=900)],
                 detector=det, layers=layers, sed_lam0=300.0, sed_dlam=1.0, sed_flux=sed_tables(temps, 300.0, 1.0, 900),
                 sersic=tables, sources=sources, atmosphere=True, sensor=True, z_entrance=ATM_Z0_MM - 1000.0)


def grad_grid_scene(n_side=8, photons=1_000_000, seed=5, zernike_nm_max=50.0):
    """The differentiation workload: 64 stars on an 8 x 8 grid over the 0.2 degree field, 1e6 photons each,
    atmosphere off; M1/M2/M3 carry Zernike Z4-Z22 figure errors drawn at 0-50 nm rms.  Returns (scene,
    params) with params = M2 and camera (lenses, filter, detector) dx, dy, tx, ty and Z4-Z22 of the three
    mirrors, as (surface, field) pairs; camera parameters apply to each of its surfaces."""
    d, surfaces, materials = three_mirror_optics()
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side) - (n_side - 1) / 2) / (n_side - 1) * math.radians(0.2)
    X, Y = np.meshgrid(g, g)
    n = X.size
    temps = rng.uniform(3000.0, 10000.0, n)
    src = point_sources(X.ravel(), Y.ravel(), np.full(n, photons, np.uint64), sed=np.arange(n))
    for m in range(3):
        s = surfaces[m]
        rms = rng.uniform(0.0, zernike_nm_max) * 1e-6
        c = rng.normal(size=19)
        c = c / np.sqrt(np.sum(c * c)) * rms
        s.zern = tuple([0.0, 0.0, 0.0] + list(c))
        s.zern_rnorm = s.r_out
    det = Detector(nx=4096, ny=4096, pixel=0.01, t_si=0.1, ell_lam0=300.0, ell_dlam=1.0,
                   ell=absorption_length_table(300.0, 1.0, 901), sigma=np.array([0.003, 0.003]))
    sc = Scene(seed=seed, pupil_r_in=d["pupil_r_in"], pupil_r_out=d["pupil_r_out"], surfaces=surfaces,
               materials=materials, coatings=[filter_coating(550.0, 700.0, 0.95, lam0=300.0, nlam=900)],
               detector=det, layers=[], sed_lam0=300.0, sed_dlam=1.0, sed_flux=sed_tables(temps, 300.0, 1.0, 900),
               sersic=np.ones((1, 4)), sources=src, atmosphere=False, sensor=True, z_entrance=ATM_Z0_MM - 1000.0)
    camera = list(range(3, len(surfaces)))
    params = [(1, f) for f in (0, 1, 3, 4)] + [(c, f) for c in camera for f in (0, 1, 3, 4)]
    params += [(m, 100 + j) for m in range(3) for j in range(3, 22)]
    return sc, params, camera


def rigid_group_pert(surfaces, group, pivot_z, dx=0.0, dy=0.0, tx=0.0, ty=0.0):
    """Per-surface misalignments (dx, dy, dz, tx, ty, tz) that move the surfaces of `group` as one rigid body
    (Sec. 2.4.1 misalignments of a whole assembly, such as the camera): the body is turned by Ry(ty) Rx(tx)
    about the point (0, 0, pivot_z), then shifted by (dx, dy).  A surface whose vertex sits h = z - pivot_z above
    the pivot keeps the body's orientation and has its vertex moved to the turned point,
    (sin ty cos tx h, -sin tx h, (cos ty cos tx - 1) h) + (dx, dy, 0).  Returns {surface: pert}."""
    out = {}
    for k in group:
        h = surfaces[k].z - pivot_z
        out[k] = (dx + math.sin(ty) * math.cos(tx) * h, dy - math.sin(tx) * h,
                  (math.cos(ty) * math.cos(tx) - 1.0) * h, tx, ty, 0.0)
    return out


def grad_grid_parameters(surfaces, params, camera, pivot_z=None):
    """The differentiation workload's enumerated parameters: M2 dx, dy, tx, ty; the camera as one rigid body
    dx, dy, tx, ty (turned about its detector vertex unless pivot_z is given); Z4-Z22 of M1, M2 and M3 (65 in
    all).  Returns (names, J) with J[i, p] the derivative of per-surface parameter params[p] (the (surface, field)
    pairs phosim_grad takes) with respect to enumerated parameter i at zero misalignment, from
    rigid_group_pert: per-surface gradients g (n_src x len(params)) give the enumerated ones as g @ J.T."""
    if pivot_z is None:
        pivot_z = surfaces[camera[-1]].z
    index = {p: k for k, p in enumerate(params)}
    names, rows = [], []

    def row(entries):
        r = np.zeros(len(params))
        for p, v in entries:
            r[index[p]] += v
        return r
    for f, nm in ((0, "dx"), (1, "dy"), (3, "tx"), (4, "ty")):
        names.append(f"M2 {nm}")
        rows.append(row([((1, f), 1.0)]))
    h = {c: surfaces[c].z - pivot_z for c in camera}
    names += ["camera dx", "camera dy", "camera tx", "camera ty"]
    rows.append(row([((c, 0), 1.0) for c in camera]))
    rows.append(row([((c, 1), 1.0) for c in camera]))
    rows.append(row([((c, 3), 1.0) for c in camera] + [((c, 1), -h[c]) for c in camera]))
    rows.append(row([((c, 4), 1.0) for c in camera] + [((c, 0), h[c]) for c in camera]))
    for m in range(3):
        for j in range(3, 22):
            names.append(f"M{m + 1} Z{j + 1}")
            rows.append(row([((m, 100 + j), 1.0)]))
    return names, np.array(rows)


# ----------------------------------------------------------------------------------------------------------
# high-frequency atmospheric kick (Sec. 2.3.2): the long-exposure PSF of the kappa > kappa_crit screens
# ----------------------------------------------------------------------------------------------------------

def structure_function_highpass(rho_m, r0_m, L0_m, f_crit):
    """Phase structure function of the part of the spectrum above f_crit (cycles/m):
    D(rho) = 4 pi int_fcrit^inf [1 - J0(2 pi f rho)] PSD(f) f df (Sec. 2.3.2, high-pass form), by quadrature on
    a logarithmic frequency grid; and the high-pass phase variance sigma^2 = 2 pi int PSD f df."""
    from scipy import special
    f = np.exp(np.linspace(math.log(f_crit), math.log(f_crit * 1e5), 200001))
    w = phase_psd(f * f, r0_m, L0_m) * f * f          # PSD f df with df = f dlnf
    dlnf = math.log(f[1] / f[0])
    rho = np.atleast_1d(np.asarray(rho_m, np.float64))
    out = np.empty_like(rho)
    for i, r in enumerate(rho):
        out[i] = 4.0 * math.pi * np.trapezoid(w * (1.0 - special.j0(2.0 * math.pi * f * r)), dx=dlnf)
    sigma2 = 2.0 * math.pi * np.trapezoid(w, dx=dlnf)
    return out, sigma2


def long_exposure_psf_radial(D_of_rho, lam_m, drho, n=2048):
    """Radially symmetric long-exposure PSF from a structure function: B(rho) = exp(-D/2) on an n x n grid of
    spacing drho, Fourier transformed; returns (theta grid of the radial profile in rad, cumulative fraction
    of the PSF within theta).  D_of_rho maps radii (m) to D."""
    x = (np.arange(n) - n // 2) * drho
    X, Y = np.meshgrid(x, x)
    R = np.hypot(X, Y)
    rr = np.unique(np.round(R.ravel() / drho * 8) / 8 * drho)
    B = np.interp(R, rr, np.exp(-0.5 * D_of_rho(rr)))
    psf = np.abs(np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(B))))
    psf /= psf.sum()
    dth = lam_m / (n * drho)
    TH = np.hypot(*np.meshgrid(x / drho * dth, x / drho * dth))
    order = np.argsort(TH.ravel())
    th = TH.ravel()[order]
    cdf = np.cumsum(psf.ravel()[order])
    return th, cdf


def fwhm_radial(D_of_rho, lam_m, drho, n=2048):
    """Full width at half maximum (rad) of the long-exposure PSF of D_of_rho."""
    x = (np.arange(n) - n // 2) * drho
    X, Y = np.meshgrid(x, x)
    R = np.hypot(X, Y)
    rr = np.unique(np.round(R.ravel() / drho * 8) / 8 * drho)
    B = np.interp(R, rr, np.exp(-0.5 * D_of_rho(rr)))
    psf = np.real(np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(B))))
    row = psf[n // 2, n // 2:] / psf[n // 2, n // 2]
    k = int(np.argmax(row < 0.5))
    frac = (row[k - 1] - 0.5) / (row[k - 1] - row[k])
    return 2.0 * (k - 1 + frac) * lam_m / (n * drho)


def high_frequency_kick_table(r0_m=0.15, L0_m=20.0, lam_ref_nm=500.0, K=4096, crit=1.5):
    """Quantiles of the kick angle (rad, at lam_ref) of the second, statistical kick of Sec. 2.3.2: the
    long-exposure PSF of the screens above kappa_crit = 2 pi / (crit r0), at u = (k + 1/2) / K.  The part
    exp(-sigma^2) of the PSF that the high-pass screens leave unscattered has zero kick."""
    lam = lam_ref_nm * 1e-9
    f_crit = 1.0 / (crit * r0_m)
    rho_tab = np.r_[0.0, np.exp(np.linspace(math.log(1e-4), math.log(50.0 * r0_m), 400))]
    D_tab, sigma2 = structure_function_highpass(rho_tab[1:], r0_m, L0_m, f_crit)
    D_tab = np.r_[0.0, D_tab]
    Dfun = lambda r: np.interp(r, rho_tab, D_tab, right=2.0 * sigma2)
    core = math.exp(-sigma2)
    drho = r0_m / 40.0
    th, cdf_total = long_exposure_psf_radial(Dfun, lam, drho)
    # the FFT of B = (B - core) + core puts the unscattered part in the central sample: remove it
    cdf_halo = np.clip((cdf_total - core) / (1.0 - core), 0.0, 1.0)
    u = (np.arange(K) + 0.5) / K
    q = np.where(u < core, 0.0, np.interp((u - core) / (1.0 - core), cdf_halo, th))
    return q, sigma2


# ----------------------------------------------------------------------------------------------------------
# charge diffusion from the silicon field model (Sec. 2.5)
# ----------------------------------------------------------------------------------------------------------

def diffusion_sigma_table(t_si_mm=0.1, v_over=20.0, T_K=173.0, n_bulk=1e12, n_b=0.0, s_b_mm=0.005, n_f=0.0,
                          s_f_mm=0.005, n=65, n_fine=4001):
    """Lateral diffusion sigma (mm) of charge converted at depths k t_si / (n - 1) below the entrance, from
    the field model of Sec. 2.5.  With z measured from the collecting (front) surface, the doping is
    n_d(z) = n_bulk + n_b exp(-(t - z) / s_b) + n_f exp(-z / s_f) (cm^-3) and the field magnitude
    E(z) = V / t + q / (eps0 eps_Si) int_z^t n_d dz' (V/cm), largest at the front.  Diffusion over the drift
    adds D dt = (mu k T / q) dz / (mu E): the mobility cancels (Einstein relation) and
    sigma^2(z_c) = 2 (k T / q) int_0^z_c dz / E(z) for charge converted at z_c."""
    q_over_eps = 1.602176634e-19 / (8.8541878128e-14 * 11.7)          # V cm
    kT_q = 8.617333262e-5 * T_K                                       # V
    t = t_si_mm * 0.1                                                  # cm
    z = np.linspace(0.0, t, n_fine)
    nd = n_bulk + n_b * np.exp(-(t - z) / (s_b_mm * 0.1)) + n_f * np.exp(-z / (s_f_mm * 0.1))
    # int_z^t n_d dz' by the trapezoid rule from the back
    seg = 0.5 * (nd[1:] + nd[:-1]) * np.diff(z)
    tail = np.r_[np.cumsum(seg[::-1])[::-1], 0.0]
    E = v_over / t + q_over_eps * tail
    inv = 1.0 / E
    cum = np.r_[0.0, np.cumsum(0.5 * (inv[1:] + inv[:-1]) * np.diff(z))]   # int_0^z dz / E
    depth = np.linspace(0.0, t, n)                                     # below the entrance (the back)
    zc = t - depth
    sig_cm = np.sqrt(2.0 * kT_q * np.interp(zc, z, cum))
    return sig_cm * 10.0                                               # mm
