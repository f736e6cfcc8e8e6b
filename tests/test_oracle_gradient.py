"""Pins of the gradient oracle (forward-mode dual numbers through the oracle's optics, Sec. 2.4):
a closed form (a decentred paraboloid still focuses on-axis light perfectly, so every photon's image moves
one-for-one with the decenter), and central differences of the oracle itself with common random numbers."""
import numpy as np

from paper_1504_06570_gb300 import inputs as I
from tests.helpers import mirror_scene
from tests import gpu_helpers as G


def test_paraboloid_decenter_moves_image_one_for_one(oracle_mod):
    sc = mirror_scene(20000.0, -1.0, 10000.0, n_photons=2000)
    o = oracle_mod.Oracle(sc)
    t = o.trace_tangents([(0, 0), (0, 1), (0, 2)])
    det = (t["flags"] & 1) == 1
    assert det.mean() > 0.99
    np.testing.assert_allclose(t["dx"][det, 0], 1.0, atol=1e-9)     # d x / d dx
    np.testing.assert_allclose(t["dy"][det, 1], 1.0, atol=1e-9)     # d y / d dy
    np.testing.assert_allclose(t["dx"][det, 1], 0.0, atol=1e-9)
    # a defocus dz of the mirror moves the focus by dz; at the fixed detector the spot grows linearly:
    # d x / d dz = +x_pupil / f for a ray at pupil height x_pupil (f = 10 m): the detector now sits dz in
    # front of the focus, where the converging ray is still on its own side of the axis
    pos, d, lam, tt = o.pre_optics(0, 0, 2000)
    np.testing.assert_allclose(t["dx"][det, 2], 2.0 * pos[det, 0] / 20000.0, rtol=2e-3, atol=1e-6)


def test_dual_numbers_match_oracle_central_differences(oracle_mod):
    counts = [400, 300]
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=2), atmosphere=False)
    params = [(0, 0), (0, 3), (1, 1), (2, 0), (5, 2), (0, 103), (0, 106), (0, 121)]
    o = oracle_mod.Oracle(sc)
    t = o.trace_tangents(params)
    for k, (si, f) in enumerate(params):
        s = sc.surfaces[si]
        h = 1e-4 if f < 3 else (1e-8 if f < 6 else 1e-7)
        outs = []
        for sgn in (1.0, -1.0):
            pert = list(s.pert) + [0.0] * (6 - len(s.pert))
            zern = list(s.zern) + [0.0] * 28
            if f < 6:
                pert[f] += sgn * h
            else:
                zern[f - 100] += sgn * h
            o.set_perturbation(si, pert, zern[:max(len(s.zern), f - 99 if f >= 100 else 0)])
            outs.append(o.trace(n_threads=4))
        o.set_perturbation(si, list(s.pert) + [0.0] * (6 - len(s.pert)), list(s.zern))
        ok = ((t["flags"] & 1) == 1) & ((outs[0]["flags"] & 1) == 1) & ((outs[1]["flags"] & 1) == 1)
        fdx = (outs[0]["x"][ok] - outs[1]["x"][ok]) / (2 * h)
        fdy = (outs[0]["y"][ok] - outs[1]["y"][ok]) / (2 * h)
        scale = max(np.abs(t["dx"][ok, k]).max(), np.abs(t["dy"][ok, k]).max(), 1e-12)
        assert np.abs(fdx - t["dx"][ok, k]).max() < 1e-5 * scale + 1e-9, (si, f)
        assert np.abs(fdy - t["dy"][ok, k]).max() < 1e-5 * scale + 1e-9, (si, f)
