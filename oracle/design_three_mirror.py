"""Design of the synthetic three-mirror survey telescope and three-lens camera used as the large workload.

The paper's telescope prescription is not part of the paper (Table 1 lists only the kinds of data), so
this script designs a stand-in of the stated size: an 8.4 m annular primary (5.1 m inner), a 3.4 m convex
secondary, a 5.0 m tertiary, three fused-silica lenses, a 550-700 nm filter and a flat detector at an
effective f/1.23.  The paraxial layout solves the focal length and back focal distance in closed form;
conic constants, low-order aspheric terms, two lens radii and the detector height are then fitted by least
squares on the RMS spot over a 0.2 degree field at three wavelengths, with the CPU oracle as raytracer.

Run: python oracle/design_three_mirror.py   (writes paper_1504_06570_gb300/data/three_mirror_camera.json)
"""
import json
import math
import os
import sys

import numpy as np
from scipy import optimize

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path[0] = ROOT            # run as a script: import the oracle package, not this folder
from oracle import oracle as O                                   # noqa: E402
from paper_1504_06570_gb300 import inputs as I                   # noqa: E402

OUT = os.path.join(ROOT, "paper_1504_06570_gb300", "data", "three_mirror_camera.json")

EFL = 10332.0            # f/1.23 on 8.4 m
R1 = 19800.0
D1 = 6100.0              # M1 -> M2
Z_FOCUS = 5400.0         # paraxial focus height (camera below the secondary)


def paraxial_radii():
    """R2, R3 from the effective focal length and the focus height (y-u ray transfer, unfolded)."""
    phi1 = 2.0 / R1
    y2 = 1.0 - D1 * phi1
    u3 = -1.0 / EFL
    y3 = Z_FOCUS / EFL
    u2 = (y3 - y2) / D1           # M2 -> M3 (M3 at the primary's vertex height)
    phi2 = (-phi1 - u2) / y2
    phi3 = (u2 - u3) / y3
    return 2.0 / phi2, 2.0 / phi3


def build(params):
    k1, k2, k3, a1_4, a2_4, a3_4, a3_6, cl3, zdet, cl1 = params
    rl1 = 1.0 / (cl1 * 1e-4) if cl1 != 0.0 else 0.0      # curvature parameters in 1e-4 / mm
    rl1b = 1.0 / (cl1 * 1.05e-4) if cl1 != 0.0 else 0.0
    rl3 = 1.0 / (cl3 * 1e-4) if cl3 != 0.0 else 0.0
    R2, R3 = paraxial_radii()
    R2, R3 = -R2, R3              # telescope frame: R > 0 puts the centre of curvature towards +z
    surfaces = [
        I.Surface(kind=I.MIRROR, R=R1, kappa=k1, alpha=(0, a1_4 * 1e-14, 0, 0, 0, 0, 0, 0), z=0.0, r_in=2550.0, r_out=4200.0),
        I.Surface(kind=I.MIRROR, R=R2, kappa=k2, alpha=(0, a2_4 * 1e-12, 0, 0, 0, 0, 0, 0), z=D1, r_in=0.0, r_out=1700.0),
        I.Surface(kind=I.MIRROR, R=R3, kappa=k3, alpha=(0, a3_4 * 1e-13, 0, a3_6 * 1e-20, 0, 0, 0, 0), z=0.0, r_in=0.0, r_out=2500.0),
        # L1: thick meniscus; L2: weak; filter plate; L3: field flattener
        I.Surface(kind=I.REFRACT, R=rl1, z=4850.0, r_out=330.0, material=1),
        I.Surface(kind=I.REFRACT, R=rl1b, z=4880.0, r_out=330.0, material=0),
        I.Surface(kind=I.REFRACT, R=-8000.0, z=5120.0, r_out=290.0, material=1),
        I.Surface(kind=I.REFRACT, R=-7000.0, z=5135.0, r_out=290.0, material=0),
        I.Surface(kind=I.REFRACT, R=0.0, z=5230.0, r_out=270.0, material=1, coating=0),
        I.Surface(kind=I.REFRACT, R=0.0, z=5240.0, r_out=270.0, material=0),
        I.Surface(kind=I.REFRACT, R=rl3, z=5300.0, r_out=260.0, material=1),
        I.Surface(kind=I.REFRACT, R=0.0, z=5325.0, r_out=260.0, material=0),
        I.Surface(kind=I.DETECTOR, R=0.0, z=zdet, material=2),
    ]
    return surfaces


MATS = [I.Material(I.VACUUM), I.Material(I.SELLMEIER, I.FUSED_SILICA_B, I.FUSED_SILICA_C), I.Material(I.SILICON)]


def scene_for(surfaces):
    det = I.Detector(nx=4096, ny=4096, pixel=0.01, t_si=0.1, ell=np.ones(2), sigma=np.zeros(2))
    return I.Scene(seed=1, pupil_r_in=2550.0, pupil_r_out=4200.0, surfaces=surfaces, materials=MATS,
                   coatings=[I.filter_coating()], detector=det, layers=[], sed_lam0=300.0, sed_dlam=1.0,
                   sed_flux=np.ones((1, 900)), sersic=np.ones((1, 4)), sources=I.point_sources([0.0], [0.0], [1]),
                   atmosphere=False, sensor=False)


def ray_bundle(theta_x, theta_y, z0, n_r=6, n_phi=16):
    r = np.sqrt(np.linspace(2600.0 ** 2, 4150.0 ** 2, n_r))
    phi = np.linspace(0, 2 * np.pi, n_phi, endpoint=False)
    R, PH = np.meshgrid(r, phi)
    x, y = (R * np.cos(PH)).ravel(), (R * np.sin(PH)).ravel()
    d = np.array([theta_x, theta_y, -math.sqrt(1 - theta_x ** 2 - theta_y ** 2)])
    t = (z0 - 0.0) / -d[2]
    pos = np.c_[x - d[0] * t, y - d[1] * t, np.full_like(x, z0)]
    return pos, np.tile(d, (len(x), 1))


FIELDS = [(0.0, 0.0), (0.05, 0.0), (0.1, 0.0), (0.0, 0.1), (0.0707, 0.0707), (0.1, 0.1)]
WAVES = [555.0, 625.0, 695.0]


def residuals(params):
    sc = scene_for(build(params))
    o = O.Oracle(sc)
    res = []
    for fx, fy in FIELDS:
        pos, d = ray_bundle(math.radians(fx), math.radians(fy), sc.z_entrance)
        xs, ys = [], []
        for lam in WAVES:
            x, y, fl = o.trace_rays(pos, d, lam)
            bad = (fl & 1) == 0
            x = np.where(bad, np.nan, x); y = np.where(bad, np.nan, y)
            xs.append(x); ys.append(y)
        X, Y = np.concatenate(xs), np.concatenate(ys)
        if np.isnan(X).any():
            res.append(np.full(2 * len(X), 1.0))
            continue
        res.append(np.r_[X - X.mean(), Y - Y.mean()])
    return np.concatenate(res)


def main():
    x0 = np.array([-1.2, -0.5, -0.2, 0.0, 0.0, 0.0, 0.0, 0.0, 5460.0, 0.0])
    # detector height first (on-axis focus), then everything together
    zs = np.linspace(5400.0, 5520.0, 121)
    def on_axis(z):
        q = x0.copy(); q[8] = z
        r = residuals(q).reshape(len(FIELDS), -1)[0]
        return np.sqrt(np.mean(r ** 2))
    x0[8] = zs[int(np.argmin([on_axis(z) for z in zs]))]
    lo = np.array([-3, -3, -3, -50, -50, -50, -50, -1.0, 5350, -1.0])
    hi = np.array([1, 1, 1, 50, 50, 50, 50, 1.0, 5560, 1.0])
    best = optimize.least_squares(residuals, x0, bounds=(lo, hi), x_scale=np.array([0.05, 0.05, 0.05, 1, 1, 1, 1, 0.2, 1.0, 0.2]),
                                  max_nfev=600)
    p = best.x
    r = residuals(p).reshape(len(FIELDS), -1)
    rms = np.sqrt(np.mean(r ** 2, axis=1) * 2)
    surfaces = build(p)
    sc = scene_for(surfaces)
    o = O.Oracle(sc)
    pos, d = ray_bundle(math.radians(0.1), 0.0, sc.z_entrance)
    x, _, _ = o.trace_rays(pos, d, 625.0)
    plate = x.mean() / 0.1          # mm per degree
    out = {
        "name": "three-mirror survey telescope with three-lens camera (synthetic stand-in)",
        "generated_by": "oracle/design_three_mirror.py",
        "efl_mm": EFL, "plate_scale_arcsec_per_mm": 3600.0 / abs(plate),
        "rms_spot_um_per_field": {f"{fx},{fy}": float(v * 1e3) for (fx, fy), v in zip(FIELDS, rms)},
        "pupil_r_in": 2550.0, "pupil_r_out": 4200.0,
        "surfaces": [{k: (list(v) if isinstance(v, (tuple, list, np.ndarray)) else v)
                      for k, v in s.__dict__.items()} for s in surfaces],
        "materials": [{"kind": m.kind, "B": list(m.B), "C": list(m.C)} for m in MATS],
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, default=float)
    print(json.dumps({k: out[k] for k in ("plate_scale_arcsec_per_mm", "rms_spot_um_per_field")}, indent=1))
    print("params", list(p))


if __name__ == "__main__":
    main()
