"""Benchmark: photons/s of the photon Monte Carlo path on one GB300 (and N GPUs by weak scaling).

Headline workload (the batched persistent launch): 10^4 sources (70 % stars, 30 % Sersic galaxies with index
0.5-4, half-light radius 0.2-3 arcsec, |e| < 0.6), photon counts log-uniform 1e2-1e7 (~8.8e9 photons), plus a
uniform sky of 1e9 photons on 15 arcsec Gaussian nodes traced as rays of 8 photons (Sec. 3.2), through seven
frozen-flow von Karman layers (4096^2 at 1 cm + 1024^2 at 64 cm each), the synthetic 8.4 m three-mirror
telescope with a three-lens camera and a 550-700 nm filter, and 100 um of silicon, onto one 4096 x 4096 chip.
A step is one phosim_trace call over all sources (autotuned schedule, dynamic transmission).  The headline is
the mixed-precision path with its FP64 parts in double-single arithmetic; the native-FP64 mixed path and the
plain all-FP64 path trace the same workload beside it, every source's moments are compared with the all-FP64
path's, and the moments of all three with the CPU oracle on a photon sample.  Extras: the 1000-star 1e8-photon
workload with the per-photon precision split, the background bundles and the adjoint.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "photons/s end-to-end on 1 GB300 vs plain FP64 path; PSF-moment error vs oracle"


def batched_name(scale=1.0, fine_n=4096, coarse_n=1024):
    return ("batched: 7000 stars + 3000 Sersic galaxies (counts log-uniform 1e2-1e7) + 1e9 sky photons on 15 arcsec "
            f"nodes in rays of 8, x{scale:g} photons; three-mirror 8.4 m telescope + 3-lens camera + 550-700 nm "
            f"filter, 7 von Karman layers ({fine_n}^2@1cm + {coarse_n}^2@64cm), 4096^2 chip")


def workload_name(photons=1e8, fine_n=4096, coarse_n=1024):
    return ("three-mirror 8.4 m telescope + 3-lens camera + 550-700 nm filter, 7 von Karman layers "
            f"({fine_n}^2@1cm + {coarse_n}^2@64cm), 1000 stars, {photons:.0e} photons, 4096^2 chip").replace("e+0", "e")


PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="photon scale of the batched workload (per GPU)")
    ap.add_argument("--plain-steps", type=int, default=2, help="timed steps of the plain FP64 path and of the "
                                                                  "native-FP64 mixed path")
    ap.add_argument("--sample", type=int, default=2000, help="oracle photons per source for the CPU leg")
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 1e8-star, background and adjoint legs")
    ap.add_argument("--stars-photons", type=float, default=1e8, help="photons of the 1000-star extra leg")
    ap.add_argument("--no-fp64-arms", action="store_true", help="time the headline path only (profiling runs)")
    ap.add_argument("--schedule", default=None, help="threads,tile for every path instead of the autotuner")
    ap.add_argument("--fine-n", type=int, default=4096, help="fine screen size (smaller: profiling case)")
    ap.add_argument("--coarse-n", type=int, default=1024, help="coarse screen size (smaller: profiling case)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; only the samples that arrive between
    mark() and stop() (the timed region) are kept."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 5.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.02)
        except OSError:
            self.proc = None

    def mark(self):
        self.t0 = time.time()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, l in self.lines:
            if self.t0 is not None and t < self.t0:
                continue
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


TRAFFIC_PROFILE = INST_PROFILE = None       # every committed summary under profiles/
KERNEL_SOURCES = ("paper_1504_06570_gb300/csrc/photon.cuh", "paper_1504_06570_gb300/csrc/trace.cu",
                  "paper_1504_06570_gb300/csrc/trace_optics.cu",
                  "paper_1504_06570_gb300/csrc/phosim_device.cuh", "paper_1504_06570_gb300/csrc/photon_ds.cuh",
                  "paper_1504_06570_gb300/csrc/ds.cuh")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _profile_records(path, tag):
    """(kernel, workload, value, photons, sources hash) of the `tag` lines of the committed ncu summaries
    (every profiles/*.md when path is None); lines without a workload field belong to the 1000-star workload."""
    import glob
    import re
    text = ""
    for f in ([path] if path else sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))):
        try:
            text += open(f).read() + "\n"
        except OSError:
            pass
    pat = tag + r": kernel=(\S+)(?: workload=(\S+))? \w+=(\d+) photons=(\d+) kernel_sources=([0-9a-f]+)"
    return [(m.group(1), m.group(2) or "stars", int(m.group(3)), int(m.group(4)), m.group(5))
            for m in re.finditer(pat, text)]


def recorded(path, tag, photons, kernel, wl):
    """A per-launch figure of a kernel (DRAM bytes or thread instructions) from a committed ncu summary, scaled
    to this launch's photons, or None when the kernel sources changed since that capture."""
    h = kernel_source_hash()
    for k, w, v, n, src in _profile_records(path, tag):
        if k == kernel and w == wl and src == h:
            return v * photons / n
    return None


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


def stars_workload(photons, fine_n=4096, coarse_n=1024):
    from paper_1504_06570_gb300 import inputs as I
    return I.three_mirror_scene(n_total=int(photons), fine_n=fine_n, coarse_n=coarse_n)


def batched_workload(scale=1.0, fine_n=4096, coarse_n=1024):
    from paper_1504_06570_gb300 import inputs as I
    return I.batched_scene(fine_n=fine_n, coarse_n=coarse_n, photon_scale=scale)


def cpu_leg(scene, sample, n_threads=None, o=None):
    """The oracle as it stands on the host cores over a bounded sample: the first `sample` photons of every
    source (all threads).  Returns its rate, its records and the per-source counts."""
    from oracle import oracle as O
    cnt = np.minimum(scene.sources.n_photons, np.uint64(sample))
    o = o or O.Oracle(scene)
    cores = n_threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    rec = o.trace(count=cnt, n_threads=cores, image=False)
    dt = time.perf_counter() - t0
    return {"value": float(cnt.sum() / dt), "unit": "photons/s", "cores": cores, "kind": "oracle",
            "sample": f"first {sample} photons of each of {len(cnt)} sources ({int(cnt.sum())} photons, {dt:.1f} s)"}, rec, cnt


def moment_errors(gpu_m, ora_rec, n_src):
    """Per-source centroid / size / ellipticity differences between the GPU sample and the oracle sample."""
    from paper_1504_06570_gb300 import phosim as P
    g = P.derived_moments(gpu_m)
    det = (ora_rec["flags"] & 1) == 1
    src = ora_rec["source"][det]
    x, y = ora_rec["x"][det], ora_rec["y"][det]
    # two-pass moments of the oracle's detected photons, per source
    n = np.bincount(src, minlength=n_src).astype(np.float64)
    ok = n >= 50
    nn = np.maximum(n, 1)
    mx, my = np.bincount(src, x, n_src) / nn, np.bincount(src, y, n_src) / nn
    dx, dy = x - mx[src], y - my[src]
    ixx, ixy, iyy = (np.bincount(src, dx * dx, n_src) / nn, np.bincount(src, dx * dy, n_src) / nn,
                     np.bincount(src, dy * dy, n_src) / nn)
    T = ixx + iyy
    gT = g[:, 3] + g[:, 5]
    with np.errstate(invalid="ignore", divide="ignore"):
        a = np.stack([np.hypot(g[:, 1] - mx, g[:, 2] - my) / np.sqrt(T), np.abs(gT / T - 1),
                      np.abs((g[:, 3] - g[:, 5]) / gT - (ixx - iyy) / T), np.abs(2 * g[:, 4] / gT - 2 * ixy / T),
                      np.abs(g[:, 0] - n) / nn], 1)[ok]
    return {"sources": int(ok.sum()), "max_centroid_over_size": float(a[:, 0].max()), "max_rel_T": float(a[:, 1].max()),
            "max_de1": float(a[:, 2].max()), "max_de2": float(a[:, 3].max()), "max_rel_count": float(a[:, 4].max())}


def moments_vs_fp64(sums, sums_fp64, min_count=100, runs=1, runs_fp64=1):
    """Every source's moments of one path against the all-FP64 path's on the same photons: worst centroid
    shift over the PSF size, relative size, e1 / e2 differences, relative detected count (the sums may hold
    several identical runs: the counts are divided by the number of runs)."""
    from paper_1504_06570_gb300 import phosim as P
    g, p = P.derived_moments(sums), P.derived_moments(sums_fp64)
    g[:, 0] /= runs
    p[:, 0] /= runs_fp64
    ok = p[:, 0] > min_count
    T, Tp = g[:, 3] + g[:, 5], p[:, 3] + p[:, 5]
    return {"sources": int(ok.sum()),
            "max_centroid_over_size": float((np.hypot(g[:, 1] - p[:, 1], g[:, 2] - p[:, 2]) / np.sqrt(Tp))[ok].max()),
            "max_rel_T": float(np.abs(T / Tp - 1)[ok].max()),
            "max_de1": float(np.abs((g[:, 3] - g[:, 5]) / T - (p[:, 3] - p[:, 5]) / Tp)[ok].max()),
            "max_de2": float(np.abs(2 * g[:, 4] / T - 2 * p[:, 4] / Tp)[ok].max()),
            "max_rel_count": float((np.abs(g[:, 0] - p[:, 0]) / np.maximum(p[:, 0], 1))[ok].max()),
            "within_0.1%": bool(np.all(np.abs(T / Tp - 1)[ok] < 1e-3))}


def algorithmic_work(sc, counts, sample=50):
    """The oracle's operation count (sums, products, quotients, roots of the FP64 program, counted by its
    operation-counting scalar on the first `sample` photons of every source, with the dynamic transmission
    test) scaled to a launch of `counts` photons.  A background bundle's ray is traced once for its photons
    (Sec. 3.2), so a bundled source's optics operations count once per ray; the entry stage's screen lookups
    are one 32-byte 2 x 2 gradient block per scale and layer for every surviving ray."""
    from oracle import oracle as O
    o = O.Oracle(sc)
    src = sc.sources
    bundle = np.ones(len(src)) if src.bundle is None else np.maximum(1, src.bundle).astype(np.float64)
    work = {"pre": {}, "optics": {}, "units": 0.0, "photons": float(np.sum(counts))}
    n_scales = sum(len(L.scales) for L in sc.layers)
    gathers = 0.0
    for b in np.unique(bundle):
        sel = bundle == b
        cnt = np.where(sel, np.minimum(counts, np.uint64(sample)), 0).astype(np.uint64)
        if cnt.sum() == 0:
            continue
        ops = o.count_ops(count=cnt, early_reject=True)
        units = float(np.sum(np.asarray(counts, np.float64)[sel]) / b)        # rays
        for part in ("pre", "optics"):
            for k, v in ops[part].items():
                work[part][k] = work[part].get(k, 0.0) + v * units
        work["units"] += units
        gathers += 32.0 * n_scales * ops["survivors"] * units
    work["gather_bytes"] = gathers
    return work


def ds_mix_peak(lib, stream, work):
    """The operation rate (Tops/s) of a path doing every one of the oracle's FP64-level operations as one
    double-single primitive, from the measured rate of each primitive (phosim_ds_rate) and the work's mix."""
    import ctypes as C
    r = C.c_double()
    rates = {}
    for name, op, it in (("add", 0, 20000), ("mul", 1, 20000), ("fma", 2, 20000), ("div", 3, 5000), ("sqrt", 4, 5000)):
        if lib.phosim_ds_rate(op, it, 4, C.c_void_p(stream), C.byref(r)) != 0:
            return None, None
        rates[name] = r.value
    mix = {k: work["optics"].get(k, 0.0) for k in ("add", "mul", "div", "sqrt")}
    t = sum(mix[k] / rates[k] for k in mix)
    return sum(mix.values()) / t, rates


def precision_split(sc, mixed, plain, counts, dev):
    """Mixed against all-FP64 on the same photons (every photon of the workload): per-photon distance of the
    final positions (pixels) for photons both detect, fate agreement, and per-star moment differences."""
    import torch
    from paper_1504_06570_gb300 import phosim as P
    n = int(counts.sum())
    d = sc.detector
    out = {}
    recs, moms = [], []
    for scn in (mixed, plain):
        rec = torch.empty(n * P.RECORD_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
        mom = torch.zeros((len(counts), P.MOMENT_WORDS), dtype=torch.float64, device=dev)
        scn.trace(img, rec, mom, n_photons=counts)
        torch.cuda.synchronize(dev)
        recs.append(rec)
        moms.append(mom.cpu().numpy())
        del img
    a, b = recs
    # 48-byte records: x, y, xc, yc, lambda (float64), flags (uint32), pixel (int32)
    xa, ya = a.view(torch.float64).view(-1, 6)[:, 0], a.view(torch.float64).view(-1, 6)[:, 1]
    xb, yb = b.view(torch.float64).view(-1, 6)[:, 0], b.view(torch.float64).view(-1, 6)[:, 1]
    fa = a.view(torch.int32).view(-1, 12)[:, 10]
    fb = b.view(torch.int32).view(-1, 12)[:, 10]
    both = ((fa & 1) == 1) & ((fb & 1) == 1)
    err = torch.maximum((xa - xb).abs(), (ya - yb).abs())[both] / d.pixel
    err, _ = torch.sort(err)
    q = lambda f: float(err[min(len(err) - 1, int(f * (len(err) - 1)))].item())
    out["photons"] = n
    out["detected_by_both"] = int(both.sum().item())
    out["fate_agreement"] = float((fa == fb).double().mean().item())
    out["position_error_px"] = {"p50": q(0.5), "p90": q(0.9), "p99": q(0.99), "p99.9": q(0.999),
                                "p99.999": q(0.99999), "max": float(err[-1].item())}
    out["per_star_vs_fp64"] = moments_vs_fp64(moms[0], moms[1])
    del recs, a, b
    torch.cuda.empty_cache()
    return out


def stars_leg(args, dev, stream):
    """The 1000-star workload (1e8 photons, the configuration of the per-photon precision split): each path
    timed, the double-single stages timed, and every photon's fate and position compared with the all-FP64
    path's."""
    import torch
    from paper_1504_06570_gb300 import phosim as P
    sc = stars_workload(args.stars_photons, args.fine_n, args.coarse_n)
    counts = sc.sources.n_photons
    n = int(counts.sum())
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
    out = {"workload": workload_name(args.stars_photons, args.fine_n, args.coarse_n), "photons_per_step": n}
    scenes = {"mixed_ds": P.Scene(sc, P.MIXED_DS, early_reject=True, graph=True),
              "mixed_fp64_optics": P.Scene(sc, P.MIXED, early_reject=True, graph=True),
              "plain_fp64": P.Scene(sc, P.PLAIN_FP64, early_reject=True)}
    for name, scn in scenes.items():
        steps = 5 if name == "mixed_ds" else 2
        scn.trace(img, None, None, stream=stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            scn.trace(img, None, None, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / steps
        out[name] = {"value": n / (ms / 1e3), "unit": "photons/s", "ms_per_step": ms}
    out["stage_ms"] = stage_times(scenes["mixed_ds"], img, None, None, None, stream, 3)
    out["precision_split"] = {"mixed_ds": precision_split(sc, scenes["mixed_ds"], scenes["plain_fp64"], counts, dev),
                              "mixed_fp64_optics": precision_split(sc, scenes["mixed_fp64_optics"],
                                                                   scenes["plain_fp64"], counts, dev)}
    for scn in scenes.values():
        scn.close()
    return out, sc


def stage_times(scene, img, mom, counts, first, stream, steps):
    """Mean milliseconds per kernel kind over `steps` traces launched kernel by kernel with CUDA events on the
    stream (the library's stage timing): chief rays, one-kernel trace, entry, optics and bundle stages."""
    import ctypes as C
    from paper_1504_06570_gb300 import phosim as P
    L = P.lib()
    L.phosim_set_stage_timing(scene.h, 1)
    acc = np.zeros(5)
    ms = (C.c_double * 5)()
    for _ in range(steps):
        scene.trace(img, None, mom, n_photons=counts, first=first, stream=stream.cuda_stream)
        if L.phosim_stage_times(scene.h, ms, 5) != 0:
            raise RuntimeError("phosim_stage_times failed")
        acc += np.array(ms[:])
    L.phosim_set_stage_timing(scene.h, 0)
    return dict(zip(("chief", "one_kernel", "entry", "optics", "bundle"), (acc / steps).tolist()))


def background_leg(layers, dev, stream, precision):
    """Sec. 3.2 background optimisation on the batched workload's sky alone (1e9 photons on 15 arcsec Gaussian
    nodes): rays of 8 photons spread by 5 arcsec on the detector against one photon per ray, timed per step,
    and the reduced chi^2 of the two images (pixel counts, (a - b)^2 / (a + b) averaged over pixels with
    counts), the statistic the paper quotes for this optimisation."""
    import torch
    from paper_1504_06570_gb300 import inputs as I
    from paper_1504_06570_gb300 import phosim as P
    out = {}
    imgs = {}
    for n in (1, 8):
        sc = I.batched_scene(fine_n=16, coarse_n=16, sky_bundle=n)
        sc.layers = layers
        sky = np.nonzero(sc.sources.kind == I.GAUSS)[0]
        sc.sources = sc.sources.subset(sky[sc.sources.n_photons[sky] > 0])
        scn = P.Scene(sc, precision, early_reject=True)
        d = sc.detector
        img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
        scn.trace(img, None, None, stream=stream.cuda_stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        img.zero_()
        a.record(stream)
        scn.trace(img, None, None, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        photons = int(sc.sources.n_photons.sum())
        out[f"photons_per_ray_{n}"] = {"value": photons / (ms / 1e3), "unit": "photons/s", "ms": ms}
        imgs[n] = img.cpu().numpy().astype(np.float64)
        scn.close()
    a, b = imgs[1], imgs[8]
    m = (a + b) > 0
    out["reduced_chi2_images"] = float(((a - b)[m] ** 2 / (a + b)[m]).mean())
    out["sky_photons_per_pixel"] = float(a.mean())
    out["speedup"] = out["photons_per_ray_8"]["value"] / out["photons_per_ray_1"]["value"]
    return out


def adjoint_leg(dev, stream):
    """Adjoint raytrace on 64 stars on an 8 x 8 grid, 1e6 photons each, no atmosphere, 97 per-surface
    parameters (M2 and each camera surface dx, dy, tx, ty; Z4-Z22 of the three mirrors), from which the 65
    enumerated ones (the camera as one rigid body) follow by a fixed Jacobian."""
    import torch
    from paper_1504_06570_gb300 import inputs as I
    from paper_1504_06570_gb300 import phosim as P
    sc, params, camera = I.grad_grid_scene()
    scn = P.Scene(sc, P.PLAIN_FP64)
    dL = np.random.default_rng(0).normal(size=(len(sc.sources), 5))
    scn.grad(dL, params)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    reps = 2
    for _ in range(reps):
        g, m = scn.grad(dL, params)
    dt = (time.perf_counter() - t0) / reps
    n = int(sc.sources.n_photons.sum())
    scn.close()
    return {"photons": n, "params": len(params), "value": n / dt, "unit": "photons/s (forward moments + adjoint)",
            "s_per_gradient": dt, "detected": int(m[:, 0].sum())}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    sc = batched_workload(args.scale, args.fine_n, args.coarse_n)
    o = O.Oracle(sc)
    steps = []
    cpu = None
    for _ in range(args.warmup + args.steps):
        cpu, _, _ = cpu_leg(sc, max(1, args.sample // 4), o=o)
        steps.append(cpu["value"])
    v = float(np.median(steps[args.warmup:]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "photons/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batched_name(args.scale, args.fine_n, args.coarse_n), "oracle_sample": cpu["sample"]},
            "cpu_baseline": {**cpu, "value": v},
            "e2e": {"value": v, "unit": "photons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import ctypes as C
    import torch
    import torch.distributed as dist
    from paper_1504_06570_gb300 import build as B
    B.build()
    from paper_1504_06570_gb300 import phosim as P
    from paper_1504_06570_gb300 import sharding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    L = P.lib()

    t_setup = time.perf_counter()
    sc = batched_workload(args.scale, args.fine_n, args.coarse_n)
    n_src = len(sc.sources)
    # weak scaling: rank r traces photons [r N, (r + 1) N) of every source (a longer exposure per GPU)
    first, counts = sharding.rank_photon_range(sc.sources.n_photons, rank, world)
    photons = int(counts.sum())
    # every path with the paper's dynamic transmission (early coating rejection), which leaves the detected
    # photons unchanged, and its launch shape picked by the autotuner on a sample of this workload
    head = P.Scene(sc, P.MIXED_DS, early_reject=True, graph=True)
    arms = {"mixed_ds": head}
    if not args.no_fp64_arms:
        arms["mixed_fp64_optics"] = P.Scene(sc, P.MIXED, early_reject=True, graph=True)
        arms["plain_fp64"] = P.Scene(sc, P.PLAIN_FP64, early_reject=True)
    tuned = {}
    for name, scn in arms.items():
        if args.schedule:
            scn.set_schedule(*[int(v) for v in args.schedule.split(",")])
            tuned[name] = scn.schedule()
        else:
            # the double-single path on 2e8 photons (~20 ms a trial): on 2e7 its trials had about three tiles
            # of 1024 photons per warp and favoured small tiles that the full workload runs slower (entry stage
            # 402 against 370 ms); the FP64 paths, 8 times slower, on 2e7
            sample = 200_000_000 if name == "mixed_ds" else 20_000_000
            tuned[name] = scn.autotune(sample_photons=sample, n_photons=counts, stream=stream.cuda_stream)
    other, plain = arms.get("mixed_fp64_optics"), arms.get("plain_fp64")
    setup_s = time.perf_counter() - t_setup
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(scene, steps, warmup, mom, on_start=None):
        for _ in range(warmup):
            scene.trace(img, None, mom, n_photons=counts, first=first, stream=stream.cuda_stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        if on_start:
            on_start()
        for a, b in ev:
            a.record(stream)
            scene.trace(img, None, mom, n_photons=counts, first=first, stream=stream.cuda_stream)
            b.record(stream)
        barrier()
        return np.array([a.elapsed_time(b) for a, b in ev])

    # peaks of the arithmetic roofline, measured on this device: FP64 and FP32 FMA rates
    fp64_rate = fp32_rate = None
    r = C.c_double()
    if L.phosim_fma_rate(1, 2000, 4, C.c_void_p(stream.cuda_stream), C.byref(r)) == 0:
        fp64_rate = r.value
    if L.phosim_fma_rate(0, 20000, 4, C.c_void_p(stream.cuda_stream), C.byref(r)) == 0:
        fp32_rate = r.value
    # ceilings of the entry stage's screen lookups: random aligned 32-byte gathers from a buffer the size of
    # the screens (HBM) and from one well inside the L2
    gather_peaks = {}
    for name, nbytes in (("hbm", 4 << 30), ("l2", 32 << 20)):
        if L.phosim_gather_rate(C.c_size_t(nbytes), 2048, 4, C.c_void_p(stream.cuda_stream), C.byref(r)) == 0:
            gather_peaks[name] = r.value

    # moment sums of each path over all its runs (warm-up and timed): the derived moments do not depend on
    # how many identical runs were added
    moms = {k: torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device=dev)
            for k in ("mixed_ds", "mixed_fp64_optics", "plain_fp64")}
    clocks = ClockSampler(local)
    clocks.start()
    per_head = timed(head, args.steps, args.warmup, moms["mixed_ds"], on_start=clocks.mark)
    clock_rec = clocks.stop()
    per_other = timed(other, args.plain_steps, 1, moms["mixed_fp64_optics"]) if other else np.array([np.nan])
    per_plain = timed(plain, args.plain_steps, 1, moms["plain_fp64"]) if plain else np.array([np.nan])
    kt = stage_times(head, img, None, counts, first, stream, 2)

    # e2e through the C ABI with host buffers: every step copies in a pinned host image (and the source list
    # and photon counts), and reads back the result image and the per-source moment sums
    himg = torch.zeros((d.ny, d.nx), dtype=torch.int32, pin_memory=True)
    dmom = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device=dev)
    hmom = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, pin_memory=True)
    head.trace(himg, None, dmom, n_photons=counts, first=first, stream=stream.cuda_stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        head.trace(himg, None, dmom, n_photons=counts, first=first, stream=stream.cuda_stream)
        hmom.copy_(dmom, non_blocking=True)
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    img_bytes = d.nx * d.ny * 4
    mom_bytes = n_src * P.MOMENT_WORDS * 8
    src_bytes = n_src * (C.sizeof(P.Source) + 16)

    t_head = float(per_head.sum()) / 1e3
    t_other = float(per_other.sum()) / 1e3
    t_plain = float(per_plain.sum()) / 1e3
    t_head, t_other, t_plain, e2e_s = sharding.max_over_ranks([t_head, t_other, t_plain, e2e_s], device=dev)
    value = photons * world * args.steps / t_head
    other_value = photons * world * args.plain_steps / t_other
    plain_value = photons * world * args.plain_steps / t_plain
    counters = head.counters()
    if not (int(counters[0]) == photons and int(counters[1]) + int(counters[2:].sum()) == photons):
        raise RuntimeError(f"headline trace accounted for {int(counters[1]) + int(counters[2:].sum())} of {photons} photons")

    # the job's image and moment sums: one sum-reduce over the ranks (photon ranges are disjoint), checked
    # against the detected counts of every rank
    img.zero_()
    job_mom = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device=dev)
    head.trace(img, None, job_mom, n_photons=counts, first=first, stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    job = sharding.reduce_job(img, job_mom, int(head.counters()[1]))

    if rank != 0:
        for scn in arms.values():
            scn.close()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    sums = {k: v.cpu().numpy() for k, v in moms.items()}
    line = {"metric": METRIC, "value": value, "unit": "photons/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_head / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2+f32", "data": "synthetic",
            "config": {"workload": batched_name(args.scale, args.fine_n, args.coarse_n),
                       "photons_per_step_per_gpu": photons, "sources": n_src,
                       "precision": "mixed, double-single (FP32-pair) positions/directions/transforms/intersections/"
                                    "wavelength, FP32 deflections/sensor",
                       "schedule": {"autotuned": tuned}, "parallelism": f"photon ranges x{world}",
                       "l2": "inputs larger than L2 (gradient screens 3.8 GB single precision, swept by the wind)",
                       "setup_s": round(setup_s, 1)},
            "mixed_fp64_optics": None if other is None else {"value": other_value, "unit": "photons/s",
                                  "ms_per_step": t_other / args.plain_steps * 1e3,
                                  "precision": "mixed, FP64 positions/directions/transforms/intersections/wavelength, "
                                               "FP32 deflections/sensor"},
            "plain_fp64": None if plain is None else {"value": plain_value, "unit": "photons/s",
                                                      "ms_per_step": t_plain / args.plain_steps * 1e3,
                                                      "speedup_of_headline": value / plain_value},
            "moments_vs_plain_fp64": None if plain is None else {
                "mixed_ds": moments_vs_fp64(sums["mixed_ds"], sums["plain_fp64"], runs=args.warmup + args.steps,
                                            runs_fp64=1 + args.plain_steps),
                "mixed_fp64_optics": moments_vs_fp64(sums["mixed_fp64_optics"], sums["plain_fp64"],
                                                     runs=1 + args.plain_steps, runs_fp64=1 + args.plain_steps)},
            "detected_fraction": float(counters[1] / max(1, counters[0])),
            "e2e": {"value": photons * world / e2e_s, "unit": "photons/s", "h2d_bytes_per_step": img_bytes + src_bytes,
                    "d2h_bytes_per_step": img_bytes + mom_bytes},
            "job_reduce": job,
            "stage_ms": kt,
            "clocks": clock_rec,
            "fma_peaks_measured_tflops": {"fp64": fp64_rate, "fp32": fp32_rate}}
    # kernels per step: chief rays, then per chunk of 2^27 photons the entry, optics and bundle stages, and
    # the moment-stripe sum
    import math
    bundle = np.ones(n_src, np.uint64) if sc.sources.bundle is None else np.maximum(1, sc.sources.bundle).astype(np.uint64)
    units = int(np.sum((counts + bundle - np.uint64(1)) // bundle))
    chunks = max(1, math.ceil(units / (1 << 27)))
    line["gpu_launches"] = (2 + 3 * chunks) * args.steps

    if not args.no_oracle:
        work = algorithmic_work(sc, counts)
        fl_opt = sum(v for k, v in work["optics"].items() if k != "transcendental")
        fl_pre = sum(v for k, v in work["pre"].items() if k != "transcendental")
        t_opt = kt["optics"] / 1e3
        achieved = fl_opt / t_opt / 1e12
        mix_peak, ds_rates = ds_mix_peak(L, stream.cuda_stream, work)
        peak32 = fp32_rate or None
        inst = recorded(INST_PROFILE, "inst_record", photons, "ds_optics_kernel", "batched")
        line["roofline"] = {
            "bound": "alu", "kernel": "ds_optics_kernel", "kernel_ms": kt["optics"], "entry_kernel_ms": kt["entry"],
            "achieved": achieved, "peak": peak32, "unit": "TFLOP/s", "frac": achieved / peak32 if peak32 else None,
            "traffic": recorded(TRAFFIC_PROFILE, "traffic_record", photons, "ds_optics_kernel", "batched"),
            "algorithmic_ops_per_launch": fl_opt,
            "note": ("achieved = the oracle's FP64-level operations of the optics and sensor (sums, products, "
                     "quotients, roots counted by its operation-counting scalar on the first 50 photons of every "
                     "source, dynamic transmission applied, a background ray counted once for its 8 photons) per "
                     "launch over the optics stage's time (CUDA events around its launches on the stream); peak = "
                     "measured FP32 FMA rate of this GPU (2 operations per instruction on the pipe the stage runs "
                     "on), the ceiling of any implementation of those operations on it"),
            "vs_double_single_emulation": {"peak_tops": mix_peak, "frac": achieved / mix_peak if mix_peak else None,
                                           "primitive_tops": ds_rates,
                                           "note": "the rate if every one of those operations were one double-single "
                                                   "primitive (measured rates, the workload's mix); above 1: the "
                                                   "stage does part of them in single precision where the error "
                                                   "budget allows"},
            "issue_frac": (inst / t_opt / 1e12) / (fp32_rate / 2) if (inst and fp32_rate) else None,
            "algorithmic_gather_bytes": work["gather_bytes"],
            "entry_gather_gbs": work["gather_bytes"] / (kt["entry"] / 1e3) / 1e9 if kt["entry"] else None,
            "hbm_peak_gbs": measured_peaks().get("hbm_gbs")}
        # the entry stage against the measured random-gather ceilings (its lookups are dependent, one per layer
        # and scale, so it sits below them: the latency of the chain, not the bandwidth, sets its time)
        g_entry = line["roofline"]["entry_gather_gbs"]
        line["roofline_entry"] = {
            "bound": "gather latency", "kernel": "ds_entry_kernel", "kernel_ms": kt["entry"], "achieved": g_entry,
            "unit": "GB/s", "peak_random_gather": gather_peaks or None,
            "frac_of_hbm_random_gather": g_entry / gather_peaks["hbm"] if (g_entry and gather_peaks.get("hbm")) else None,
            "note": "achieved = algorithmic bytes of the screen lookups (32 B per layer and scale of every surviving "
                    "ray) over the entry stage's time; peaks = phosim_gather_rate: independent random aligned "
                    "32-byte gathers from a 4 GiB buffer (HBM) and a 32 MiB one (L2) on this device"}
        # native-FP64 mixed kernel: the same operations against the FP64 FMA rate
        peak64 = fp64_rate or FP64_NOMINAL_TFLOPS
        if other is not None:
            kt_other = stage_times(other, img, None, counts, first, stream, 1)
            line["roofline_mixed_fp64_optics"] = {
                "bound": "alu", "kernel": "trace_kernel<1>", "kernel_ms": kt_other["one_kernel"],
                "achieved": fl_opt / (kt_other["one_kernel"] / 1e3) / 1e12, "peak": peak64, "unit": "TFLOP/s",
                "note": "the oracle's optics operations per launch over the kernel's time; peak = " +
                        ("measured FP64 FMA rate" if fp64_rate else "nominal FP64 (fallback)")}
            line["roofline_mixed_fp64_optics"]["frac"] = line["roofline_mixed_fp64_optics"]["achieved"] / peak64
        if plain is not None:
            line["roofline_plain_fp64"] = {"achieved": (fl_opt + fl_pre) / (t_plain / args.plain_steps) / 1e12,
                                           "peak": peak64, "unit": "TFLOP/s"}
            line["roofline_plain_fp64"]["frac"] = line["roofline_plain_fp64"]["achieved"] / peak64
        cpu, rec, cnt = cpu_leg(sc, args.sample)
        line["cpu_baseline"] = cpu
        errs = {}
        for name, scn in arms.items():
            m2 = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device=dev)
            i2 = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
            scn.trace(i2, None, m2, n_photons=cnt)
            torch.cuda.synchronize(dev)
            errs[name] = moment_errors(m2.cpu().numpy(), rec, n_src)
        line["moment_error_vs_oracle"] = errs
    for scn in arms.values():
        scn.close()
    if not args.no_extras:
        line["stars_1e8"], sc_stars = stars_leg(args, dev, stream)
        line["background_bundles"] = background_leg(sc_stars.layers, dev, stream, P.MIXED_DS)
        line["adjoint"] = adjoint_leg(dev, stream)
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
