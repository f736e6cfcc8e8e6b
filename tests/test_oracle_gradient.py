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


def test_tilt_and_zernike_gradients_closed_forms(oracle_mod):
    """Sec. 2.4.1 misalignments and figure, differentiated: a vertical beam on a flat mirror reaches the
    detector plane z = L above it at y = y0 - tan(2 tx)(L - y0 tan tx) and x = x0 + tan(2 ty)(L + x0 tan ty)
    (exact trigonometry), so at zero tilt dy/dtx = -2 L and dx/dty = +2 L for every photon.  A Noll Z2 term
    of coefficient c over rho_n is the plane z = (2 c / rho_n) x, which turns the beam by twice its slope:
    dx/dc = -4 L / rho_n at c = 0 (Z3 likewise in y).  With c != 0 and the mirror turned by tz the spot is
    (x0, y0) + (L - z_h) s (cos tz, sin tz), s = -2 g / (1 - g^2), g = 2 c / rho_n, z_h = g (x0 cos tz + y0 sin
    tz), so at tz = 0: dx/dtz = -g y0 s and dy/dtz = (L - g x0) s."""
    from tests.test_oracle_pins import _flat_mirror_scene
    L, rn = 500.0, 1000.0
    src = I.point_sources([0.0], [0.0], [1500])
    sc = _flat_mirror_scene(zern=(0.0, 0.0, 0.0), rnorm=rn, L=L, sources=src)
    o = oracle_mod.Oracle(sc)
    t = o.trace_tangents([(0, 3), (0, 4), (0, 101), (0, 102)])
    det = (t["flags"] & 1) == 1
    assert det.mean() > 0.99
    np.testing.assert_allclose(t["dy"][det, 0], -2 * L, rtol=1e-12)
    np.testing.assert_allclose(t["dx"][det, 0], 0.0, atol=1e-9)
    np.testing.assert_allclose(t["dx"][det, 1], 2 * L, rtol=1e-12)
    np.testing.assert_allclose(t["dy"][det, 1], 0.0, atol=1e-9)
    np.testing.assert_allclose(t["dx"][det, 2], -4 * L / rn, rtol=1e-12)
    np.testing.assert_allclose(t["dy"][det, 2], 0.0, atol=1e-12)
    np.testing.assert_allclose(t["dy"][det, 3], -4 * L / rn, rtol=1e-12)
    np.testing.assert_allclose(t["dx"][det, 3], 0.0, atol=1e-12)
    c = 0.3
    g = 2 * c / rn
    s = -2 * g / (1 - g * g)
    sc = _flat_mirror_scene(zern=(0.0, c), rnorm=rn, L=L, sources=src)
    o = oracle_mod.Oracle(sc)
    t = o.trace_tangents([(0, 5)])
    det = (t["flags"] & 1) == 1
    pos, _, _, _ = o.pre_optics(0, 0, 1500)
    x0, y0 = pos[det, 0], pos[det, 1]
    np.testing.assert_allclose(t["dx"][det, 0], -g * y0 * s, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(t["dy"][det, 0], (L - g * x0) * s, rtol=1e-9, atol=1e-12)
