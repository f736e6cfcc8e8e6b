"""The adjoint raytrace (phosim_grad) against the oracle's forward-mode dual numbers (an exact derivative of
the same program) and against central finite differences of the CUDA forward pass with common random
numbers.  The oracle comparison is tight (1e-6 relative: both are exact derivatives evaluated in FP64 in a
different order); finite differences carry truncation error and photons crossing accept boundaries, so
they are held to 1e-3 of the gradient's scale."""
import numpy as np
import pytest

from paper_1504_06570_gb300 import inputs as I
from paper_1504_06570_gb300 import phosim as P
from tests import gpu_helpers as G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

PARAMS = [(0, 0), (0, 1), (0, 3), (0, 4), (1, 0), (1, 1), (2, 0), (5, 2), (5, 0), (0, 103), (0, 104), (0, 106),
          (0, 110), (0, 121)]


def oracle_gradient(oracle_mod, scene, dL, params):
    o = oracle_mod.Oracle(scene)
    t = o.trace_tangents(params, n_threads=8)
    n_src = len(scene.sources)
    g = np.zeros((n_src, len(params)))
    det = (t["flags"] & 1) == 1
    for s in range(n_src):
        m = det & (t["source"] == s)
        n = m.sum()
        if n == 0:
            continue
        x, y = t["x"][m], t["y"][m]
        dx, dy = x - x.mean(), y - y.mean()
        fx = dL[s, 0] / n + 2 * dL[s, 2] / n * dx + dL[s, 3] / n * dy
        fy = dL[s, 1] / n + 2 * dL[s, 4] / n * dy + dL[s, 3] / n * dx
        g[s] = fx @ t["dx"][m] + fy @ t["dy"][m]
    return g


def scene_for_grad(counts, seed=2, sensor=True):
    sc = G.test_system_scene(sources=G.mixed_sources(counts, seed=seed), atmosphere=False, sensor=sensor)
    return sc


@pytest.mark.parametrize("sensor", [True, False])
def test_adjoint_matches_oracle_forward_mode(oracle_mod, sensor):
    counts = [3000, 1500, 2500, 33]
    sc = scene_for_grad(counts, sensor=sensor)
    rng = np.random.default_rng(1)
    dL = rng.normal(size=(len(counts), 5))
    s = P.Scene(sc, P.PLAIN_FP64)
    g, m = s.grad(dL, PARAMS)
    s.close()
    go = oracle_gradient(oracle_mod, sc, dL, PARAMS)
    scale = np.abs(go).max(axis=0) + 1e-300
    err = np.abs(g - go) / scale
    assert err.max() < 1e-6, (err.max(axis=0), g[0], go[0])


def test_adjoint_matches_central_differences():
    counts = [4000, 2000, 3000]
    sc = scene_for_grad(counts, seed=7)
    rng = np.random.default_rng(3)
    dL = rng.normal(size=(len(counts), 5))
    s = P.Scene(sc, P.PLAIN_FP64)
    g, _ = s.grad(dL, PARAMS)
    base = {p: (sc.surfaces[p[0]].pert[p[1]] if p[1] < 6 else
                (sc.surfaces[p[0]].zern[p[1] - 100] if p[1] - 100 < len(sc.surfaces[p[0]].zern) else 0.0))
            for p in PARAMS}
    scales = {0: 1.0, 1: 1.0, 2: 1.0, 3: 1e-4, 4: 1e-4, 5: 1e-4}
    for k, p in enumerate(PARAMS):
        h = 1e-3 * (scales[p[1]] if p[1] < 6 else 1e-4)
        vals = []
        for sgn in (1, -1):
            s.set_parameters([p], [base[p] + sgn * h])
            _, m = s.grad(np.zeros((len(counts), 5)), PARAMS)
            vals.append((dL * m[:, 1:]).sum(axis=1))
        s.set_parameters([p], [base[p]])
        fd = (vals[0] - vals[1]) / (2 * h)
        tol = 1e-3 * (np.abs(g[:, k]).max() + 1e-12)
        assert np.all(np.abs(fd - g[:, k]) <= tol), (p, fd, g[:, k])
    s.close()


def test_autograd_function_backward_is_the_adjoint():
    counts = [2000, 1000]
    sc = scene_for_grad(counts, seed=5)
    s = P.Scene(sc, P.PLAIN_FP64)
    params = [(0, 3), (1, 0), (0, 103)]
    theta = torch.tensor([2e-6, 0.05, 3e-5], dtype=torch.float64, requires_grad=True)
    M = P.psf_moments(theta, s, params)
    w = torch.tensor(np.random.default_rng(0).normal(size=tuple(M.shape)))
    (M * w).sum().backward()
    g, _ = s.grad(w.numpy(), params)
    np.testing.assert_allclose(theta.grad.numpy(), g.sum(0), rtol=1e-12)
    s.close()


def test_autograd_forward_is_one_trace_with_the_adjoints_moments():
    """The forward pass of PSFMoments is a single FP64 trace with moment sums; its moments are those of the
    adjoint's own forward pass (same photons, same FP64 kernel), derived by phosim_moments_derive."""
    counts = [2000, 1000, 0]
    sc = scene_for_grad(counts, seed=6)
    s = P.Scene(sc, P.PLAIN_FP64)
    params = [(0, 3), (1, 0)]
    theta = torch.tensor([1e-6, 0.02], dtype=torch.float64)
    M = P.psf_moments(theta, s, params).numpy()
    _, m = s.grad(np.zeros((len(counts), 5)), params)
    np.testing.assert_allclose(M[:2], m[:2, 1:], rtol=1e-12, atol=1e-15)
    assert np.all(M[2] == 0)          # a source with no photons has no moments (NaN mapped to 0)
    with pytest.raises(ValueError):
        P.psf_moments(theta, P.Scene(sc, P.MIXED_DS), params)
    s.close()
