"""Benchmark: photons/s of the photon Monte Carlo path on one GB300 (and N GPUs by weak scaling).

Workload: 1000 stars, 1e8 source photons per step (300-1200 nm blackbodies) through seven frozen-flow von
Karman layers (4096^2 at 1 cm + 1024^2 at 64 cm each), the synthetic 8.4 m three-mirror telescope with a
three-lens camera and a 550-700 nm filter, and 100 um of silicon, onto one 4096 x 4096 chip.  A step is one
phosim_trace call over all photons.  The headline is the mixed-precision path with its FP64 parts in
double-single arithmetic (--mode ds, the default) or in native FP64 (--mode mixed); the other mixed form and
the plain all-FP64 path are timed beside it, and the moments of all three are compared with the CPU oracle on
a photon sample.

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
def workload_name(photons=1e8, fine_n=4096, coarse_n=1024):
    return ("three-mirror 8.4 m telescope + 3-lens camera + 550-700 nm filter, 7 von Karman layers "
            f"({fine_n}^2@1cm + {coarse_n}^2@64cm), 1000 stars, {photons:.0e} photons, 4096^2 chip").replace("e+0", "e")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--photons", type=float, default=1e8, help="photons per step per GPU")
    ap.add_argument("--mode", default="ds", choices=["ds", "mixed"], help="headline mixed-precision form")
    ap.add_argument("--plain-steps", type=int, default=3, help="timed steps of the plain FP64 path and of the "
                                                                  "other mixed form")
    ap.add_argument("--sample", type=int, default=8000, help="oracle photons per star for the CPU leg")
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the precision-split, batched and adjoint legs")
    ap.add_argument("--batched-scale", type=float, default=1.0, help="photon scale of the batched workload")
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


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "launches_three_mirror_1e8.md")
KERNEL_SOURCES = ("paper_1504_06570_gb300/csrc/photon.cuh", "paper_1504_06570_gb300/csrc/trace.cu",
                  "paper_1504_06570_gb300/csrc/phosim_device.cuh", "paper_1504_06570_gb300/csrc/photon_ds.cuh",
                  "paper_1504_06570_gb300/csrc/ds.cuh")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def recorded_traffic(photons, kernel):
    """DRAM bytes per launch of a trace kernel (trace_kernel<1> native-FP64 mixed, ds_optics_kernel the
    double-single optics stage) from the committed ncu summary, scaled to this launch's photons, or None when
    the kernel sources changed since that capture."""
    import re
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    for m in re.finditer(r"traffic_record: kernel=(\S+) bytes=(\d+) photons=(\d+) kernel_sources=([0-9a-f]+)", text):
        if m.group(1) == kernel and m.group(4) == kernel_source_hash():
            return int(m.group(2)) * photons / int(m.group(3))
    return None


INST_PROFILE = os.path.join(ROOT, "profiles", "ds_stages_three_mirror_2e7.md")


def recorded_instructions(photons, kernel):
    """Thread instructions one launch of a kernel executes (ncu smsp__inst_executed x threads per instruction on
    the committed capture), scaled to this launch's photons, or None when the kernel sources changed since."""
    import re
    try:
        text = open(INST_PROFILE).read()
    except OSError:
        return None
    for m in re.finditer(r"inst_record: kernel=(\S+) thread_inst=(\d+) photons=(\d+) kernel_sources=([0-9a-f]+)", text):
        if m.group(1) == kernel and m.group(4) == kernel_source_hash():
            return int(m.group(2)) * photons / int(m.group(3))
    return None


# FP32 instructions of each double-single primitive of ds.cuh (sum: TwoSum 6 + 2 + Fast2Sum 3; product:
# 1 multiply + 3 FMAs + Fast2Sum 3; quotient: reciprocal estimate, product, ds x float product 6, ds sum 11,
# correction and Fast2Sum; square root: reciprocal-root estimate, product, exact square, ds sum, correction)
DS_INSTRUCTIONS = {"add": 11, "mul": 7, "div": 23, "sqrt": 20}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


def workload(photons_per_gpu, rank, fine_n=4096, coarse_n=1024):
    from paper_1504_06570_gb300 import inputs as I
    return I.three_mirror_scene(n_total=int(photons_per_gpu), fine_n=fine_n, coarse_n=coarse_n)


def cpu_leg(scene, sample):
    """The oracle as it stands on the host cores over a bounded sample: the first `sample` photons of every
    star (all threads).  Returns its rate and its records for the moment comparison."""
    from oracle import oracle as O
    cnt = np.minimum(scene.sources.n_photons, np.uint64(sample))
    o = O.Oracle(scene)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    rec = o.trace(count=cnt, n_threads=cores, image=False)
    dt = time.perf_counter() - t0
    return {"value": float(cnt.sum() / dt), "unit": "photons/s", "cores": cores, "kind": "oracle",
            "sample": f"first {sample} photons of each of {len(cnt)} stars ({int(cnt.sum())} photons, {dt:.1f} s)"}, rec, cnt


def moment_errors(gpu_m, ora_rec, n_src):
    """Per-star centroid / size / ellipticity differences between the GPU sample and the oracle sample."""
    from paper_1504_06570_gb300 import phosim as P
    g = P.derived_moments(gpu_m)
    det = (ora_rec["flags"] & 1) == 1
    out = []
    for s in range(n_src):
        m = det & (ora_rec["source"] == s)
        if m.sum() < 50:
            continue
        x, y = ora_rec["x"][m], ora_rec["y"][m]
        mx, my = x.mean(), y.mean()
        ixx, ixy, iyy = ((x - mx) ** 2).mean(), ((x - mx) * (y - my)).mean(), ((y - my) ** 2).mean()
        T = ixx + iyy
        gT = g[s, 3] + g[s, 5]
        out.append([abs(g[s, 1] - mx) / np.sqrt(T), abs(gT / T - 1), abs((g[s, 3] - g[s, 5]) / gT - (ixx - iyy) / T),
                    abs(2 * g[s, 4] / gT - 2 * ixy / T), abs(g[s, 0] - m.sum()) / m.sum()])
    a = np.array(out)
    return {"stars": len(a), "max_centroid_over_size": float(a[:, 0].max()), "max_rel_T": float(a[:, 1].max()),
            "max_de1": float(a[:, 2].max()), "max_de2": float(a[:, 3].max()), "max_rel_count": float(a[:, 4].max())}


def gather_bytes_per_launch(sc, ops, photons):
    """Algorithmic screen bytes: one 32-byte 2 x 2 gradient block per scale and layer for every photon that
    survives the dynamic transmission test (fraction from the oracle's count, photons with no work)."""
    n_scales = sum(len(L.scales) for L in sc.layers)
    surv = ops.get("survivors", None)
    frac = surv if surv is not None else 1.0
    return int(32 * n_scales * frac * photons)


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
    gm, gp = P.derived_moments(moms[0]), P.derived_moments(moms[1])
    T = gp[:, 3] + gp[:, 5]
    ok = gp[:, 0] > 100
    e1m = (gm[:, 3] - gm[:, 5]) / (gm[:, 3] + gm[:, 5]); e1p = (gp[:, 3] - gp[:, 5]) / T
    e2m = 2 * gm[:, 4] / (gm[:, 3] + gm[:, 5]); e2p = 2 * gp[:, 4] / T
    out["per_star_vs_fp64"] = {"stars": int(ok.sum()), "max_de1": float(np.abs(e1m - e1p)[ok].max()),
                               "max_de2": float(np.abs(e2m - e2p)[ok].max()),
                               "max_rel_size": float(np.abs((gm[:, 3] + gm[:, 5]) / T - 1)[ok].max()),
                               "max_centroid_px": float(np.hypot(gm[:, 1] - gp[:, 1], gm[:, 2] - gp[:, 2])[ok].max() / d.pixel)}
    del recs, a, b
    torch.cuda.empty_cache()
    return out


def batched_leg(sc2, args, dev, stream, precision):
    """10^4 stars and Sersic galaxies with counts log-uniform 1e2-1e7 plus 1e9 sky photons on 15 arcsec
    Gaussian nodes (rays of 8 photons, Sec. 3.2), one persistent launch per step with the autotuned schedule
    (same optics and atmosphere)."""
    import torch
    from paper_1504_06570_gb300 import inputs as I
    from paper_1504_06570_gb300 import phosim as P
    t0 = time.perf_counter()
    sc = I.batched_scene(fine_n=16, coarse_n=16, photon_scale=args.batched_scale)
    sc.layers = sc2.layers
    scn = P.Scene(sc, precision, early_reject=True)
    threads, tile = scn.autotune(sample_photons=20_000_000)
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
    mom = torch.zeros((len(sc.sources), P.MOMENT_WORDS), dtype=torch.float64, device=dev)
    scn.trace(img, None, mom, stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    steps = 2
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        scn.trace(img, None, mom, stream=stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    n = int(sc.sources.n_photons.sum())
    c = scn.counters()
    if not (int(c[0]) == n and int(c[1]) + int(c[2:].sum()) == n):
        raise RuntimeError(f"batched trace accounted for {int(c[1]) + int(c[2:].sum())} of {n} photons")
    scn.close()
    kinds = np.bincount(sc.sources.kind, minlength=3)
    return {"workload": f"{kinds[0]} stars + {kinds[1]} Sersic galaxies (counts log-uniform 1e2-1e7) + {kinds[2]} "
                        f"sky nodes (1e9 photons in rays of 8), x{args.batched_scale} photons", "photons_per_step": n,
            "value": n / (ms / 1e3), "unit": "photons/s", "ms_per_step": ms, "autotuned": {"threads": threads, "tile": tile},
            "setup_s": round(time.perf_counter() - t0, 1)}


def background_leg(sc2, dev, stream, precision):
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
        sc.layers = sc2.layers
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
    parameters (M2 and each camera surface dx, dy, tx, ty; Z4-Z22 of the three mirrors)."""
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
    sc = workload(args.photons, 0, args.fine_n, args.coarse_n)
    steps = []
    cpu = None
    for _ in range(args.warmup + args.steps):
        cpu, _, _ = cpu_leg(sc, max(1, args.sample // 4))
        steps.append(cpu["value"])
    v = float(np.median(steps[args.warmup:]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "photons/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.photons, args.fine_n, args.coarse_n), "oracle_sample": cpu["sample"]},
            "cpu_baseline": {**cpu, "value": v},
            "e2e": {"value": v, "unit": "photons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_1504_06570_gb300 import build as B
    B.build()
    from paper_1504_06570_gb300 import phosim as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    t_setup = time.perf_counter()
    sc = workload(args.photons, rank, args.fine_n, args.coarse_n)
    n_src = len(sc.sources)
    # weak scaling: rank r traces photons [r N, (r + 1) N) of every star (a longer exposure per GPU)
    from paper_1504_06570_gb300 import sharding
    first, counts = sharding.rank_photon_range(sc.sources.n_photons, rank, world)
    photons = int(counts.sum())
    # every path with the paper's dynamic transmission (early coating rejection), which leaves the detected
    # photons unchanged; the headline form as a CUDA graph
    head_prec, other_prec = (P.MIXED_DS, P.MIXED) if args.mode == "ds" else (P.MIXED, P.MIXED_DS)
    head = P.Scene(sc, head_prec, early_reject=True, graph=True)
    other = P.Scene(sc, other_prec, early_reject=True, graph=True)
    plain = P.Scene(sc, P.PLAIN_FP64, early_reject=True)
    setup_s = time.perf_counter() - t_setup
    d = sc.detector
    img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
    mom = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(scene, steps, warmup, on_start=None):
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
        per = np.array([a.elapsed_time(b) for a, b in ev])
        return per

    # peaks of the arithmetic roofline (FMA issue rate), measured on this device
    fp64_rate = fp32_rate = None
    try:
        import ctypes as C
        r = C.c_double()
        if P.lib().phosim_fma_rate(1, 2000, 4, C.c_void_p(stream.cuda_stream), C.byref(r)) == 0:
            fp64_rate = r.value
        if P.lib().phosim_fma_rate(0, 20000, 4, C.c_void_p(stream.cuda_stream), C.byref(r)) == 0:
            fp32_rate = r.value
    except Exception:
        pass

    def kernel_times(scene, steps):
        """Mean milliseconds per kernel kind (chief rays, one-kernel trace, entry stage, optics stage) over
        `steps` traces launched kernel by kernel with CUDA events on the stream (the library's stage timing)."""
        import ctypes as C
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
        return acc / steps

    clocks = ClockSampler(local)
    clocks.start()
    per_head = timed(head, args.steps, args.warmup, on_start=clocks.mark)
    clock_rec = clocks.stop()
    per_other = timed(other, args.plain_steps, 1)
    per_plain = timed(plain, args.plain_steps, 1)
    kt_head = kernel_times(head, 3)
    kt_other = kernel_times(other, 2)

    # e2e through the C ABI with host buffers: pinned host image in, result image out, every step
    himg = torch.zeros((d.ny, d.nx), dtype=torch.int32, pin_memory=True)
    for _ in range(1):
        head.trace(himg, None, None, n_photons=counts, first=first, stream=stream.cuda_stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        head.trace(himg, None, None, n_photons=counts, first=first, stream=stream.cuda_stream)
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    img_bytes = d.nx * d.ny * 4
    src_bytes = n_src * (P.C.sizeof(P.Source) if hasattr(P, "C") else 80) + n_src * 16

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

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    names = {P.MIXED_DS: "mixed_ds", P.MIXED: "mixed_fp64_optics"}
    descr = {P.MIXED_DS: "mixed, double-single (FP32-pair) positions/directions/transforms/intersections/wavelength, "
                         "FP32 deflections/sensor",
             P.MIXED: "mixed, FP64 positions/directions/transforms/intersections/wavelength, FP32 deflections/sensor"}
    line = {"metric": METRIC, "value": value, "unit": "photons/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_head / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32x2+f32" if head_prec == P.MIXED_DS else "f64+f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.photons, args.fine_n, args.coarse_n),
                       "photons_per_step_per_gpu": photons, "sources": n_src,
                       "precision": descr[head_prec],
                       "l2": "inputs larger than L2 (gradient screens 2.8 GB, read in both precisions' forms)",
                       "setup_s": round(setup_s, 1)},
            names[other_prec]: {"value": other_value, "unit": "photons/s",
                                "ms_per_step": t_other / args.plain_steps * 1e3, "precision": descr[other_prec]},
            "plain_fp64": {"value": plain_value, "unit": "photons/s", "ms_per_step": t_plain / args.plain_steps * 1e3,
                           "speedup_of_headline": value / plain_value},
            "detected_fraction": float(counters[1] / max(1, counters[0])),
            "e2e": {"value": photons * world / e2e_s, "unit": "photons/s", "h2d_bytes_per_step": img_bytes + src_bytes,
                    "d2h_bytes_per_step": img_bytes},
            # per step: chief rays, then the entry and optics stages and the moment-stripe sum (double-single)
            # or the one trace kernel
            "gpu_launches": (4 if head_prec == P.MIXED_DS else 2) * args.steps, "clocks": clock_rec,
            "fma_peaks_measured_tflops": {"fp64": fp64_rate, "fp32": fp32_rate}}

    if not args.no_oracle:
        from oracle import oracle as O
        o = O.Oracle(sc)
        ops = o.count_ops(count=np.minimum(counts, np.uint64(50)), early_reject=True)
        fl_pre = sum(v for k, v in ops["pre"].items() if k != "transcendental")
        fl_opt = sum(v for k, v in ops["optics"].items() if k != "transcendental")
        kt_mixed = kt_head if head_prec == P.MIXED else kt_other
        kt_ds = kt_head if head_prec == P.MIXED_DS else kt_other
        peak64 = fp64_rate or FP64_NOMINAL_TFLOPS
        # native-FP64 mixed kernel (one kernel): the oracle's FP64 optics flops against the FP64 FMA rate
        fp64_roof = {"bound": "alu", "kernel": "trace_kernel<1>", "kernel_ms": float(kt_mixed[1]),
                     "achieved": fl_opt * photons / (float(kt_mixed[1]) / 1e3) / 1e12,
                     "peak": peak64, "unit": "TFLOP/s", "traffic": recorded_traffic(photons, "trace_kernel<1>"),
                     "note": (f"FP64 optics flops {fl_opt:.0f} per sampled photon (oracle op count with the dynamic "
                              f"transmission rejection; +{fl_pre:.0f} sampling and atmosphere flops, mostly FP32 "
                              f"here) over the kernel's time (CUDA events around its launches on the stream); peak = "
                              + ("measured FP64 FMA rate" if fp64_rate else "nominal FP64 (fallback)"))}
        fp64_roof["frac"] = fp64_roof["achieved"] / peak64
        # double-single kernel: bound by FP32 instruction issue.  achieved = the thread instructions the optics
        # stage executes per launch (committed ncu capture, per sampled photon) over its time; peak = the SMs'
        # issue rate (measured FP32 FMA rate / 2: one FMA a lane a cycle).  The oracle's FP64 operations over
        # the same time give the emulated FP64 rate, against the native FP64 FMA rate.
        peak32 = fp32_rate / 2 if fp32_rate else None
        t_opt = float(kt_ds[3]) / 1e3
        inst = recorded_instructions(photons, "ds_optics_kernel")
        ds_inst = sum(ops["optics"][k] * c for k, c in DS_INSTRUCTIONS.items())
        emulated = fl_opt * photons / t_opt / 1e12
        ds_roof = {"bound": "alu", "kernel": "ds_optics_kernel", "kernel_ms": float(kt_ds[3]),
                   "entry_kernel_ms": float(kt_ds[2]),
                   "achieved": inst / t_opt / 1e12 if inst else None,
                   "peak": peak32, "unit": "Tinst/s", "traffic": recorded_traffic(photons, "ds_optics_kernel"),
                   "instructions_per_photon": inst / photons if inst else None,
                   "note": ("thread instructions of the optics stage per sampled photon (ncu smsp__inst_executed x "
                            "threads per instruction on the committed 2e7-photon capture of the same kernel "
                            "sources, profiles/ds_stages_three_mirror_2e7.md) x photons over the stage's time (CUDA "
                            "events around its launches on the stream); peak = measured FP32 FMA rate / 2, the issue "
                            "rate of one instruction a lane a cycle"),
                   "emulated_fp64": {"tflops": emulated, "vs_measured_fp64_peak": emulated / peak64,
                                     "note": (f"the oracle's FP64 optics operations per sampled photon ({fl_opt:.0f}: "
                                              f"{ops['optics']['add']:.0f} add, {ops['optics']['mul']:.0f} mul, "
                                              f"{ops['optics']['div']:.0f} div, {ops['optics']['sqrt']:.0f} sqrt; "
                                              f"{ds_inst:.0f} FP32 instructions as double-single primitives "
                                              f"{DS_INSTRUCTIONS}) over the optics stage's time")}}
        ds_roof["frac"] = ds_roof["achieved"] / peak32 if (peak32 and inst) else None
        head_roof, other_roof = (ds_roof, fp64_roof) if head_prec == P.MIXED_DS else (fp64_roof, ds_roof)
        head_roof["algorithmic_gather_bytes"] = gather_bytes_per_launch(sc, ops, photons)
        head_roof["traffic_unit"] = "DRAM bytes per launch (ncu, committed summary)"
        line["roofline"] = head_roof
        line["roofline_" + names[other_prec]] = other_roof
        line["roofline_plain_fp64"] = {"achieved": (fl_opt + fl_pre) * photons / (float(np.mean(per_plain)) / 1e3) / 1e12,
                                       "peak": peak64, "unit": "TFLOP/s"}
        line["roofline_plain_fp64"]["frac"] = line["roofline_plain_fp64"]["achieved"] / peak64
        if rank == 0:
            cpu, rec, cnt = cpu_leg(sc, args.sample)
            line["cpu_baseline"] = cpu
            errs = {}
            for name, scn in ((names[head_prec], head), (names[other_prec], other), ("plain_fp64", plain)):
                m2 = torch.zeros((n_src, P.MOMENT_WORDS), dtype=torch.float64, device=dev)
                i2 = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
                scn.trace(i2, None, m2, n_photons=cnt)
                torch.cuda.synchronize(dev)
                errs[name] = moment_errors(m2.cpu().numpy(), rec, n_src)
            line["moment_error_vs_oracle"] = errs
    if not args.no_extras and rank == 0:
        line["precision_split"] = {names[head_prec]: precision_split(sc, head, plain, counts, dev),
                                   names[other_prec]: precision_split(sc, other, plain, counts, dev)}
        line["batched"] = batched_leg(sc, args, dev, stream, head_prec)
        line["background_bundles"] = background_leg(sc, dev, stream, head_prec)
        line["adjoint"] = adjoint_leg(dev, stream)
    print(json.dumps(line))
    head.close()
    other.close()
    plain.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
