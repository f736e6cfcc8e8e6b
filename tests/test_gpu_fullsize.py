"""Parity at the full size of the large workload, in the launch configuration the benchmark times (1000 stars,
1e8 photons, 4096^2 + 1024^2 screens on 7 layers, early rejection, default schedule): the oracle recomputes
a random block of 64 photons of every star one by one, and properties that hold at any size are checked on
all 1e8 photons (the image is the histogram of the detected records; every photon is accounted for)."""
import numpy as np
import pytest

from paper_1504_06570_gb300 import inputs as I
from paper_1504_06570_gb300 import phosim as P
from tests import gpu_helpers as G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def scene():
    return I.three_mirror_scene()


@pytest.mark.parametrize("precision", [P.PLAIN_FP64, P.MIXED, P.MIXED_DS])
def test_full_size_sampled_parity(oracle_mod, scene, precision):
    sc = scene
    counts = sc.sources.n_photons
    n = int(counts.sum())
    s = P.Scene(sc, precision, early_reject=True, graph=(precision != P.PLAIN_FP64))
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    rec = torch.zeros(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
    s.trace(img, rec, mom)
    torch.cuda.synchronize()
    c = s.counters()
    s.close()
    # every photon accounted for; the image is the histogram of the detected records
    assert c[0] == n and c[0] == c[1] + c[2:].sum()
    r32 = rec.view(torch.int32).view(-1, 12)
    flags, pix = r32[:, 10], r32[:, 11]
    det = (flags & 1) == 1
    assert int(det.sum().item()) == int(c[1])
    hist = torch.bincount(pix[det].long(), minlength=d.nx * d.ny)
    assert torch.equal(hist.to(torch.int32), img.view(-1))
    # a random block of 64 photons of every star, recomputed by the oracle
    rng = np.random.default_rng(17)
    first = (rng.random(len(counts)) * (counts - 64).astype(np.float64)).astype(np.uint64)
    block = np.full(len(counts), 64, np.uint64)
    ora = G.oracle_trace(oracle_mod, sc, n_photons=block, first=first)
    off = np.r_[0, np.cumsum(counts)[:-1]].astype(np.int64)
    idx = (off[:, None] + first.astype(np.int64)[:, None] + np.arange(64)[None, :]).ravel()
    sample = P.records_to_numpy(rec.view(-1, P.RECORD_DTYPE.itemsize)[torch.as_tensor(idx, device="cuda")].reshape(-1))
    gpu = {"rec": sample}
    bnd = G.boundary_mask(ora)
    det_g = (sample["flags"] & 1) == 1
    det_o = (ora["flags"] & 1) == 1
    assert np.all((det_g == det_o) | bnd)
    both = det_g & det_o
    err = np.maximum(np.abs(sample["x"][both] - ora["x"][both]), np.abs(sample["y"][both] - ora["y"][both])) / d.pixel
    if precision == P.PLAIN_FP64:
        assert np.mean(err <= 1e-4) >= 0.99999 and err.max() < 1e-4, err.max()
        okpix = both & ~bnd
        assert np.array_equal(sample["pix"][okpix], ora["pix"][okpix])
    else:
        assert np.mean(err < 1e-2) > 0.999, np.percentile(err, [50, 99, 100])


def test_double_single_chunks_compose():
    """A double-single launch larger than one chunk of the state buffer (2^27 photons) runs the entry and optics
    stages chunk after chunk, each with its own state and batch counts: 1.5e8 photons in one call must give
    exactly the image and counts of two calls over complementary photon ranges of every source, each of which
    fits one chunk, and every photon is counted once."""
    sc = I.three_mirror_scene(n_total=150_000_000, fine_n=256, coarse_n=64)
    counts = sc.sources.n_photons.astype(np.uint64)
    n = int(counts.sum())
    assert n > (1 << 27)
    s = P.Scene(sc, P.MIXED_DS, early_reject=True)
    d = sc.detector

    def run(cnt, first=None):
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        s.trace(img, None, None, n_photons=cnt, first=first)
        torch.cuda.synchronize()
        return img.cpu().numpy().view(np.uint32), s.counters()

    full, c_full = run(counts)
    a = counts // np.uint64(2)
    part1, c1 = run(a)
    part2, c2 = run(counts - a, first=a)
    s.close()
    assert int(c_full[0]) == n and int(c_full[1]) + int(c_full[2:].sum()) == n
    assert np.array_equal(c_full, c1 + c2)
    assert np.array_equal(full, part1 + part2)
    assert int(full.sum()) == int(c_full[1])
