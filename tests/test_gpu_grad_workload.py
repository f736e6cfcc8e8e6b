"""The adjoint raytrace at the differentiation workload's own scale: 64 stars on an 8 x 8 grid over the 0.2 degree
field of the three-mirror telescope, atmosphere off, Z4-Z22 figure errors of 0-50 nm rms on M1, M2 and M3 (the
workload traces 1e6 photons per star; here 2e4 per star for the finite differences and 256 per star for the
oracle, for run time).  The 65 enumerated parameters are M2 dx, dy, tx, ty; the camera (three lenses, the filter
and the detector) as one rigid body dx, dy, tx, ty turned about its detector vertex; and Z4-Z22 of the three
mirrors.  phosim_grad returns per-surface gradients (97 here) and the enumerated ones follow by the Jacobian of
the rigid-body motion (inputs.grad_grid_parameters).

- Against the oracle's forward-mode dual numbers (an exact derivative of the same FP64 program, evaluated in a
  different order): 1e-6 of each parameter's gradient scale.
- Against central differences of the CUDA FP64 forward pass with common random numbers, each parameter stepped by
  1e-3 of its scale (1 mm for decenters, 1e-4 rad for tilts, 50 nm for Zernike coefficients) and the camera moved
  by the exact rigid-body formula (inputs.rigid_group_pert), which checks the Jacobian's pivot terms: 1e-3 of the
  gradient's scale (finite differences also see photons that cross an accept boundary)."""
import numpy as np
import pytest

from paper_1504_06570_gb300 import inputs as I
from paper_1504_06570_gb300 import phosim as P

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

PHOTONS_FD = 20_000
PHOTONS_ORACLE = 256


@pytest.fixture(scope="module")
def workload():
    sc, params, camera = I.grad_grid_scene(photons=PHOTONS_FD)
    names, J = I.grad_grid_parameters(sc.surfaces, params, camera)
    assert len(names) == 65 and J.shape == (65, len(params))
    dL = np.random.default_rng(8).normal(size=(len(sc.sources), 5))
    return sc, params, camera, names, J, dL


def test_workload_gradient_matches_oracle_dual_numbers(oracle_mod, workload):
    sc, params, camera, names, J, dL = workload
    n_src = len(sc.sources)
    cnt = np.full(n_src, PHOTONS_ORACLE, np.uint64)
    s = P.Scene(sc, P.PLAIN_FP64)
    g, m = s.grad(dL, params, n_photons=cnt)
    s.close()
    t = oracle_mod.Oracle(sc).trace_tangents(params, count=cnt, n_threads=16)
    go = np.zeros((n_src, len(params)))
    det = (t["flags"] & 1) == 1
    for k in range(n_src):
        sel = det & (t["source"] == k)
        n = sel.sum()
        assert n == m[k, 0]
        x, y = t["x"][sel], t["y"][sel]
        dx, dy = x - x.mean(), y - y.mean()
        fx = dL[k, 0] / n + 2 * dL[k, 2] / n * dx + dL[k, 3] / n * dy
        fy = dL[k, 1] / n + 2 * dL[k, 4] / n * dy + dL[k, 3] / n * dx
        go[k] = fx @ t["dx"][sel] + fy @ t["dy"][sel]
    G, Go = g @ J.T, go @ J.T
    scale = np.abs(Go).max(axis=0)
    assert np.all(scale > 0)
    err = np.abs(G - Go) / scale
    assert err.max() < 1e-6, (names[int(np.argmax(err.max(axis=0)))], err.max())


def test_workload_gradient_matches_central_differences(workload):
    sc, params, camera, names, J, dL = workload
    n_src = len(sc.sources)
    s = P.Scene(sc, P.PLAIN_FP64)
    g, _ = s.grad(dL, params)
    G = g @ J.T
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    sums = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device="cuda")

    def loss():
        sums.zero_()
        s.trace(img, None, sums)
        m = P.derived_moments(sums)
        return (dL * m[:, 1:]).sum(axis=1)

    pivot = sc.surfaces[camera[-1]].z
    zero = {c: (0.0,) * 6 for c in camera}

    def set_camera(pert):
        pairs, vals = [], []
        for c, p in pert.items():
            for f in range(6):
                pairs.append((c, f)); vals.append(p[f])
        s.set_parameters(pairs, vals)

    for i, name in enumerate(names):
        part, kind = name.split()
        if kind.startswith("Z"):
            step = 1e-3 * 5e-5
        elif kind in ("dx", "dy"):
            step = 1e-3 * 1.0
        else:
            step = 1e-3 * 1e-4
        vals = []
        for sgn in (1.0, -1.0):
            h = sgn * step
            if part == "camera":
                set_camera(I.rigid_group_pert(sc.surfaces, camera, pivot, **{kind: h}))
            elif part == "M2" and not kind.startswith("Z"):
                s.set_parameters([(1, {"dx": 0, "dy": 1, "tx": 3, "ty": 4}[kind])], [h])
            else:
                m_ = int(part[1]) - 1
                j = int(kind[1:]) - 1
                base = sc.surfaces[m_].zern[j]
                s.set_parameters([(m_, 100 + j)], [base + h])
            vals.append(loss())
            # back to the nominal design
            if part == "camera":
                set_camera(zero)
            elif part == "M2" and not kind.startswith("Z"):
                s.set_parameters([(1, {"dx": 0, "dy": 1, "tx": 3, "ty": 4}[kind])], [0.0])
            else:
                s.set_parameters([(m_, 100 + j)], [base])
        fd = (vals[0] - vals[1]) / (2 * step)
        tol = 1e-3 * (np.abs(G[:, i]).max() + 1e-300)
        assert np.all(np.abs(fd - G[:, i]) <= tol), (name, np.abs(fd - G[:, i]).max(), tol)
    s.close()
