"""Small scene builders shared by the tests (inputs only, no per-photon arithmetic)."""
import numpy as np

from paper_1504_06570_gb300 import inputs as I


def bare_scene(surfaces, materials=None, coatings=None, nx=256, pixel=0.01, n_photons=1000, seed=1, sed_T=5800.0,
               lam_lo=400.0, lam_hi=700.0, sensor=False, atmosphere=False, layers=None, pupil=(0.0, 500.0),
               sources=None, t_si=0.1, sigma=0.003):
    nb = int(round(lam_hi - lam_lo))
    det = I.Detector(nx=nx, ny=nx, pixel=pixel, t_si=t_si, ell_lam0=lam_lo, ell_dlam=1.0,
                     ell=I.absorption_length_table(lam_lo, 1.0, nb + 1), sigma=np.array([sigma, sigma]))
    src = sources if sources is not None else I.point_sources([0.0], [0.0], [n_photons])
    return I.Scene(seed=seed, pupil_r_in=pupil[0], pupil_r_out=pupil[1], surfaces=surfaces,
                   materials=materials or [I.Material(I.VACUUM), I.Material(I.SILICON)], coatings=coatings or [],
                   detector=det, layers=layers or [], sed_lam0=lam_lo, sed_dlam=1.0,
                   sed_flux=I.sed_tables([sed_T], lam_lo, 1.0, nb), sersic=np.ones((1, 4)), sources=src,
                   atmosphere=atmosphere, sensor=sensor)


def mirror_scene(R, kappa, focus_z, r_out=500.0, **kw):
    surfaces = [I.Surface(kind=I.MIRROR, R=R, kappa=kappa, z=0.0, r_in=0.0, r_out=r_out),
                I.Surface(kind=I.DETECTOR, R=0.0, z=focus_z, material=1)]
    return bare_scene(surfaces, **kw)
