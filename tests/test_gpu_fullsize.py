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
    # per-star moments of the same sampled photons (those both detect), GPU records against oracle records:
    # the 0.1 % moment gate for every precision
    src = np.repeat(np.arange(len(counts)), 64)
    worst = 0.0
    for s_ in range(len(counts)):
        k = both & (src == s_)
        if k.sum() < 5:
            continue
        xg, yg, xo, yo = sample["x"][k], sample["y"][k], ora["x"][k], ora["y"][k]
        To = xo.var() + yo.var()
        for a, b in ((xg.mean(), xo.mean()), (yg.mean(), yo.mean())):
            worst = max(worst, abs(a - b) / np.sqrt(To))
        for a, b in ((xg.var(), xo.var()), (yg.var(), yo.var()),
                     (((xg - xg.mean()) * (yg - yg.mean())).mean(), ((xo - xo.mean()) * (yo - yo.mean())).mean())):
            worst = max(worst, abs(a - b) / To)
    assert worst < 1e-3, worst


def test_precision_split_full_workload():
    """Each mixed path against the all-FP64 GPU path on every one of the 1e8 photons of the large workload: the
    photons keep the all-FP64 fate (at most 1e-7 of them differ, at accept boundaries), the positions of photons
    both detect agree to 1e-4 pixel at the 99.999th percentile, and every star's centroid, size and ellipticity
    agree within the 0.1 % moment gate."""
    sc = I.three_mirror_scene()
    counts = sc.sources.n_photons
    n = int(counts.sum())
    d = sc.detector
    recs, sums = {}, {}
    for prec in (P.PLAIN_FP64, P.MIXED, P.MIXED_DS):
        s = P.Scene(sc, prec, early_reject=True)
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        rec = torch.empty(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
        s.trace(img, rec, mom)
        torch.cuda.synchronize()
        s.close()
        del img
        r = rec.view(torch.float64).view(-1, 6)
        recs[prec] = (r[:, 0].clone(), r[:, 1].clone(), rec.view(torch.int32).view(-1, 12)[:, 10].clone())
        sums[prec] = mom.cpu().numpy()
        del rec, r
        torch.cuda.empty_cache()
    xp, yp, fp = recs[P.PLAIN_FP64]
    gp = P.derived_moments(sums[P.PLAIN_FP64])
    ok = gp[:, 0] > 100
    Tp = gp[:, 3] + gp[:, 5]
    for prec in (P.MIXED, P.MIXED_DS):
        x, y, f = recs[prec]
        assert int((f != fp).sum().item()) <= n // 10_000_000
        both = ((f & 1) == 1) & ((fp & 1) == 1)
        err = torch.maximum((x - xp).abs(), (y - yp).abs())[both] / d.pixel
        q = torch.quantile(err[torch.randperm(len(err), device=err.device)[:10_000_000]].double(), 0.99999).item()
        assert q <= 1e-4, q
        g = P.derived_moments(sums[prec])
        T = g[:, 3] + g[:, 5]
        assert np.all(np.abs(np.hypot(g[:, 1] - gp[:, 1], g[:, 2] - gp[:, 2]) / np.sqrt(Tp))[ok] < 1e-3)
        assert np.all(np.abs(T / Tp - 1)[ok] < 1e-3)
        assert np.all(np.abs((g[:, 3] - g[:, 5]) / T - (gp[:, 3] - gp[:, 5]) / Tp)[ok] < 1e-3)
        assert np.all(np.abs(2 * g[:, 4] / T - 2 * gp[:, 4] / Tp)[ok] < 1e-3)


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


@pytest.fixture(scope="module")
def batched():
    return I.batched_scene()


def _batched_sample(sc, seed=31):
    """A fixed sample of the batched workload's sources: one Sersic galaxy of every index level (64), 96 stars
    and 48 sky nodes (rays of 8 photons), with a block of 64 photons of each at a random offset."""
    rng = np.random.default_rng(seed)
    src = sc.sources
    ser = np.nonzero(src.kind == I.SERSIC)[0]
    pick = [int(rng.choice(ser[src.table[ser] == t])) for t in np.unique(src.table[ser])]
    pick += list(rng.choice(np.nonzero(src.kind == I.POINT)[0], 96, replace=False))
    pick += list(rng.choice(np.nonzero(src.kind == I.GAUSS)[0], 48, replace=False))
    pick = np.array(sorted(pick))
    cnt = np.zeros(len(src), np.uint64)
    first = np.zeros(len(src), np.uint64)
    cnt[pick] = 64
    first[pick] = (rng.random(len(pick)) * (src.n_photons[pick] - 64).astype(np.float64)).astype(np.uint64)
    return pick, cnt, first


def test_batched_workload_full_launch_and_sampled_parity(oracle_mod, batched):
    """The batched workload (10^4 stars and Sersic galaxies with counts log-uniform 1e2-1e7, plus 1e9 sky photons
    in rays of 8) in the launch configuration the benchmark times (double-single, early rejection, CUDA graph,
    autotuned schedule): every photon of the full launch is accounted for and the image holds the detected
    ones; then a fixed sample of sources (every Sersic index level, stars, sky nodes) is traced photon by photon
    in every precision and compared with the oracle: fates identical away from flagged accept boundaries,
    positions within 1e-4 pixel (FP64) or 1e-2 pixel for 99.9 % of photons (mixed paths)."""
    sc = batched
    counts = sc.sources.n_photons
    n = int(counts.sum())
    d = sc.detector
    s = P.Scene(sc, P.MIXED_DS, early_reject=True, graph=True)
    s.autotune(sample_photons=20_000_000)
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
    s.trace(img)
    torch.cuda.synchronize()
    c = s.counters()
    assert int(c[0]) == n and int(c[1]) + int(c[2:].sum()) == n
    assert int(img.sum().item()) == int(c[1])
    pick, cnt, first = _batched_sample(sc)
    ora = G.oracle_trace(oracle_mod, sc, n_photons=cnt, first=first)
    bnd = G.boundary_mask(ora)
    det_o = (ora["flags"] & 1) == 1
    assert det_o.sum() > 1000
    for prec in (P.MIXED_DS, P.MIXED, P.PLAIN_FP64):
        scn = s if prec == P.MIXED_DS else P.Scene(sc, prec, early_reject=True)
        m = int(cnt.sum())
        rec = torch.zeros(m * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        i2 = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        scn.trace(i2, rec, None, n_photons=cnt, first=first)
        torch.cuda.synchronize()
        r = P.records_to_numpy(rec)
        if prec != P.MIXED_DS:
            scn.close()
        det_g = (r["flags"] & 1) == 1
        assert np.all((det_g == det_o) | bnd), prec
        # losses agree too, except that the dynamic transmission test reports a photon it rejects as a
        # coating loss even where the oracle (no early test) finds an earlier surface vignetting it
        reason_g, reason_o = (r["flags"] >> 8) & 0xFF, (ora["flags"] >> 8) & 0xFF
        early = (reason_g == 5) & (reason_o != 5) & ~det_o
        assert np.all((r["flags"] == ora["flags"]) | bnd | early), prec
        both = det_g & det_o
        err = np.maximum(np.abs(r["x"][both] - ora["x"][both]), np.abs(r["y"][both] - ora["y"][both])) / d.pixel
        if prec == P.PLAIN_FP64:
            assert np.mean(err <= 1e-4) >= 0.99999 and err.max() < 1e-4, err.max()
        else:
            assert np.mean(err < 1e-2) > 0.999, np.percentile(err, [50, 99, 100])
        kinds = sc.sources.kind[ora["source"][both]]
        assert set(np.unique(kinds)) == {I.POINT, I.SERSIC, I.GAUSS}
    s.close()


def test_batched_workload_moments_double_single_vs_fp64(batched):
    """Equal moment accuracy on the batched workload: every source's moments from the double-single path (the
    benchmark's headline) and from the all-FP64 path over all ~9.8e9 photons agree within the 0.1 % gate
    (centroid within 1e-3 of the size, size and ellipticities within 1e-3), for sources with > 100 detected
    photons, and the detected counts agree to 1e-6."""
    sc = batched
    d = sc.detector
    out = {}
    for prec in (P.MIXED_DS, P.PLAIN_FP64):
        s = P.Scene(sc, prec, early_reject=True)
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        mom = torch.zeros((len(sc.sources), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
        s.trace(img, None, mom)
        torch.cuda.synchronize()
        s.close()
        out[prec] = P.derived_moments(mom)
    g, gp = out[P.MIXED_DS], out[P.PLAIN_FP64]
    ok = gp[:, 0] > 100
    assert ok.sum() > 5000
    assert np.all(np.abs(g[:, 0] - gp[:, 0]) <= 1e-6 * gp[:, 0] + 1)
    T, Tp = g[:, 3] + g[:, 5], gp[:, 3] + gp[:, 5]
    assert np.all((np.hypot(g[:, 1] - gp[:, 1], g[:, 2] - gp[:, 2]) / np.sqrt(Tp))[ok] < 1e-3)
    assert np.all(np.abs(T / Tp - 1)[ok] < 1e-3)
    assert np.all(np.abs((g[:, 3] - g[:, 5]) / T - (gp[:, 3] - gp[:, 5]) / Tp)[ok] < 1e-3)
    assert np.all(np.abs(2 * g[:, 4] / T - 2 * gp[:, 4] / Tp)[ok] < 1e-3)


def test_multi_chunk_launch_as_one_graph():
    """PHOSIM_GRAPH with a launch of several chunks of the state buffer (2^27 work units each): the whole call
    (chief rays; per chunk the counter resets, the entry, optics and bundle stages; the moment-stripe sum) is one
    CUDA graph, rebuilt when the number of chunks or the kernel list changes and otherwise replayed with the
    call's parameters.  Every call gives the image, counters and moment sums of the same call launched kernel by
    kernel: two calls in a row on the batched workload (1.95e8 photons, sky in rays of 8, two chunks), a
    one-chunk call, and the two-chunk call again."""
    sc = I.batched_scene(fine_n=256, coarse_n=64, photon_scale=0.02)
    counts = sc.sources.n_photons.astype(np.uint64)
    d = sc.detector
    ref = P.Scene(sc, P.MIXED_DS, early_reject=True)
    gr = P.Scene(sc, P.MIXED_DS, early_reject=True, graph=True)

    def run(s, cnt):
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device="cuda")
        mom = torch.zeros((len(cnt), P.MOMENT_WORDS), dtype=torch.float64, device="cuda")
        s.trace(img, None, mom, n_photons=cnt)
        torch.cuda.synchronize()
        return img.cpu().numpy(), s.counters(), mom.cpu().numpy()

    small = np.minimum(counts, np.uint64(2000))
    bundle = np.maximum(1, sc.sources.bundle).astype(np.uint64)
    units = int(((counts + bundle - np.uint64(1)) // bundle).sum())
    assert units > (1 << 27) and int(small.sum()) < (1 << 27)
    for cnt in (counts, counts, small, counts):
        a, b = run(ref, cnt), run(gr, cnt)
        assert np.array_equal(a[0], b[0])
        assert np.array_equal(a[1], b[1])
        assert int(b[1][0]) == int(cnt.sum()) and int(b[1][1]) == int(b[0].sum())
        np.testing.assert_allclose(b[2], a[2], rtol=1e-12, atol=1e-12)
    ref.close()
    gr.close()
