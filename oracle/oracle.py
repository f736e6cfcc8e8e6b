"""ctypes front end of the CPU oracle (phosim_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's CPU-baseline leg.
It marshals a scene from paper_1504_06570_gb300.inputs into the oracle's own data layout; nothing here
computes any step of the photon path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "phosim_oracle.cpp")
LIB = os.path.join(HERE, "_build", "libphosim_oracle.so")
_lock = threading.Lock()
_lib = None

F_DETECTED = 1


def build(force=False):
    """Compile the oracle with g++ (FP contraction off so that summation order is the written one)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = f"{LIB}.{os.getpid()}.tmp"     # concurrent builders each write their own file; the replace is atomic
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            vp, d, i, u64 = C.c_void_p, C.c_double, C.c_int, C.c_uint64
            P = np.ctypeslib.ndpointer
            L.oracle_new.restype = vp
            L.oracle_new.argtypes = [u64, d, d, d, d, d, i, i]
            L.oracle_free.argtypes = [vp]
            L.oracle_index.restype = d
            L.oracle_index.argtypes = [vp, i, d]
            _lib = L
    return _lib


def _dp(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(C.POINTER(C.c_double))


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Oracle:
    """The oracle's copy of one scene."""

    def __init__(self, scene):
        L = lib()
        self.L = L
        self.scene = scene
        self.h = C.c_void_p(L.oracle_new(C.c_uint64(scene.seed), scene.pupil_r_in, scene.pupil_r_out, scene.h_top,
                                         scene.z_entrance, scene.lambda_ref, int(scene.atmosphere), int(scene.sensor)))
        self._keep = []
        for m in scene.materials:
            L.oracle_add_material(self.h, C.c_int(m.kind), _dp(m.B), _dp(m.C))
        self._coat_keep = []
        for c in scene.coatings:
            T = _arr(c.table, np.float64)
            R = getattr(c, "reflect", None)
            R = None if R is None else _arr(R, np.float64)
            self._coat_keep.append((T, R))
            L.oracle_add_coating(self.h, C.c_double(c.lam0), C.c_double(c.dlam), C.c_double(c.theta0),
                                 C.c_double(c.dtheta), C.c_int(T.shape[0]), C.c_int(T.shape[1]), _dp(T),
                                 None if R is None else _dp(R))
        for s in scene.surfaces:
            self._add_surface(s)
        d = scene.detector
        ell = _arr(d.ell, np.float64)
        sig = _arr(d.sigma, np.float64)
        L.oracle_set_detector(self.h, C.c_int(d.nx), C.c_int(d.ny), C.c_double(d.pixel), C.c_double(d.x0),
                              C.c_double(d.y0), C.c_double(d.t_si), C.c_double(d.ell_lam0), C.c_double(d.ell_dlam),
                              C.c_int(len(ell)), _dp(ell), C.c_int(len(sig)), _dp(sig))
        for layer in scene.layers:
            k = L.oracle_add_layer(self.h, C.c_double(layer.z), C.c_double(layer.vx), C.c_double(layer.vy))
            for sc in layer.scales:
                ph = _arr(sc.phase, np.float64)
                L.oracle_add_scale(self.h, C.c_int(k), C.c_double(sc.pixel), C.c_int(ph.shape[0]), _dp(ph))
        flux = _arr(scene.sed_flux, np.float64)
        L.oracle_set_seds(self.h, C.c_double(scene.sed_lam0), C.c_double(scene.sed_dlam), C.c_int(flux.shape[0]),
                          C.c_int(flux.shape[1]), _dp(flux))
        sr = _arr(scene.sersic, np.float64)
        L.oracle_set_sersic(self.h, C.c_int(sr.shape[0]), C.c_int(sr.shape[1]), _dp(sr))
        L.oracle_set_sensor_options(self.h, C.c_int(int(getattr(scene, "back_reflect", False))),
                                    C.c_double(float(getattr(scene.detector, "dead_layer", 0.0))))
        L.oracle_set_fringe(self.h, C.c_int(int(getattr(scene, "fringe", False))),
                            C.c_double(float(getattr(scene.detector, "t_si_gx", 0.0))),
                            C.c_double(float(getattr(scene.detector, "t_si_gy", 0.0))))
        if getattr(scene, "hf_kick", None) is not None and len(scene.hf_kick):
            hf = _arr(scene.hf_kick, np.float64)
            L.oracle_set_hf_kick(self.h, C.c_int(len(hf)), _dp(hf))

    def _add_surface(self, s):
        alpha = np.zeros(8)
        alpha[:len(s.alpha)] = s.alpha
        pert = np.zeros(6)
        pert[:len(s.pert)] = s.pert
        zern = _arr(s.zern if len(s.zern) else [0.0], np.float64)
        self.L.oracle_add_surface(self.h, C.c_int(s.kind), C.c_double(s.R), C.c_double(s.kappa), _dp(alpha),
                                  C.c_double(s.z), C.c_double(s.r_in), C.c_double(s.r_out), C.c_int(s.material),
                                  C.c_int(s.coating), _dp(pert), C.c_double(s.zern_rnorm), C.c_int(len(s.zern)),
                                  _dp(zern))

    def set_perturbation(self, surface, pert, zern):
        pert = _arr(pert, np.float64)
        zern = _arr(zern if len(zern) else [0.0], np.float64)
        self.L.oracle_set_perturbation(self.h, C.c_int(surface), _dp(pert), C.c_int(len(zern)), _dp(zern))

    def __del__(self):
        try:
            self.L.oracle_free(self.h)
        except Exception:
            pass

    def _src_args(self, src):
        a = [_arr(src.kind, np.int32), _arr(src.sed, np.int32), _arr(src.table, np.int32)]
        b = [_arr(getattr(src, k), np.float64) for k in ("xi", "eta", "redshift", "t0", "t_exp", "a", "b", "pa")]
        self._keep = a + b
        ip = C.POINTER(C.c_int)
        return [x.ctypes.data_as(ip) for x in a] + [x.ctypes.data_as(C.POINTER(C.c_double)) for x in b]

    def trace(self, sources=None, first=None, count=None, n_threads=1, image=True):
        """Trace photons [first[s], first[s] + count[s]) of every source; returns a dict of per-photon
        records (concatenated in source order) and the image."""
        src = self.scene.sources if sources is None else sources
        n = len(src)
        first = np.zeros(n, np.uint64) if first is None else _arr(first, np.uint64)
        count = _arr(src.n_photons if count is None else count, np.uint64)
        tot = int(count.sum())
        rec = {k: np.zeros(tot) for k in ("x", "y", "xc", "yc", "lam", "margin_mm", "margin_nm")}
        rec["flags"] = np.zeros(tot, np.uint32)
        rec["pix"] = np.zeros(tot, np.int32)
        det = self.scene.detector
        img = np.zeros((det.ny, det.nx), np.uint32) if image else None
        u64p = C.POINTER(C.c_uint64)
        dp = C.POINTER(C.c_double)
        bn = _arr(getattr(src, "bundle", None) if getattr(src, "bundle", None) is not None else np.ones(n), np.int32)
        bs = _arr(getattr(src, "bundle_sigma", None) if getattr(src, "bundle_sigma", None) is not None else np.zeros(n),
                  np.float64)
        self._keep_b = (bn, bs)
        self.L.oracle_set_bundles(self.h, C.c_int(n), bn.ctypes.data_as(C.POINTER(C.c_int)), _dp(bs))
        rc = self.L.oracle_trace(self.h, C.c_int(n), *self._src_args(src), first.ctypes.data_as(u64p),
                                 count.ctypes.data_as(u64p), *(rec[k].ctypes.data_as(dp) for k in ("x", "y", "xc", "yc", "lam")),
                                 rec["flags"].ctypes.data_as(C.POINTER(C.c_uint32)),
                                 rec["pix"].ctypes.data_as(C.POINTER(C.c_int32)),
                                 rec["margin_mm"].ctypes.data_as(dp), rec["margin_nm"].ctypes.data_as(dp),
                                 None if img is None else img.ctypes.data_as(C.POINTER(C.c_uint32)), C.c_int(n_threads))
        if rc != 0:
            raise RuntimeError(f"oracle_trace failed ({rc})")
        rec["source"] = np.repeat(np.arange(n), count.astype(np.int64))
        rec["index"] = np.concatenate([np.arange(int(f), int(f) + int(c), dtype=np.uint64) for f, c in zip(first, count)]) if n else np.zeros(0, np.uint64)
        rec["image"] = img
        return rec

    def trace_rays(self, pos, dirs, lam):
        pos = _arr(pos, np.float64).reshape(-1, 3)
        dirs = _arr(dirs, np.float64).reshape(-1, 3)
        lam = _arr(np.broadcast_to(lam, (len(pos),)), np.float64)
        n = len(pos)
        ox, oy = np.zeros(n), np.zeros(n)
        fl = np.zeros(n, np.uint32)
        self.L.oracle_trace_rays(self.h, C.c_int(n), _dp(pos), _dp(dirs), _dp(lam), _dp(ox), _dp(oy), None, None,
                                 fl.ctypes.data_as(C.POINTER(C.c_uint32)))
        return ox, oy, fl

    def intersect(self, surface, pos, d):
        l = C.c_double()
        hit, nrm = np.zeros(3), np.zeros(3)
        rc = self.L.oracle_intersect(self.h, C.c_int(surface), _dp(pos), _dp(d), C.byref(l), _dp(hit), _dp(nrm))
        return rc, l.value, hit, nrm

    def sag(self, surface, x, y):
        x = _arr(x, np.float64); y = _arr(y, np.float64)
        z, zx, zy = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
        self.L.oracle_sag(self.h, C.c_int(surface), C.c_int(len(x)), _dp(x), _dp(y), _dp(z), _dp(zx), _dp(zy))
        return z, zx, zy

    def index(self, material, lam_nm):
        return self.L.oracle_index(self.h, C.c_int(material), C.c_double(lam_nm))

    def cdf(self, sed):
        out = np.zeros(self.scene.sed_flux.shape[1])
        self.L.oracle_get_cdf(self.h, C.c_int(sed), _dp(out))
        return out

    def pre_optics(self, src_index, first, count, sources=None):
        src = self.scene.sources if sources is None else sources
        pos, d = np.zeros((count, 3)), np.zeros((count, 3))
        lam, t = np.zeros(count), np.zeros(count)
        rc = self.L.oracle_pre_optics(self.h, C.c_int(len(src)), *self._src_args(src), C.c_int(src_index),
                                      C.c_uint64(first), C.c_uint64(count), _dp(pos), _dp(d), _dp(lam), _dp(t))
        if rc:
            raise RuntimeError("oracle_pre_optics failed")
        return pos, d, lam, t

    def count_ops(self, sources=None, first=None, count=None, early_reject=False):
        """Algorithmic operations per sampled photon: dict of sampling+atmosphere and optics+sensor counts.
        early_reject: photons the dynamic transmission test drops before propagation count no operations."""
        src = self.scene.sources if sources is None else sources
        n = len(src)
        first = np.zeros(n, np.uint64) if first is None else _arr(first, np.uint64)
        count = _arr(src.n_photons if count is None else count, np.uint64)
        out = np.zeros(12)
        u64p = C.POINTER(C.c_uint64)
        rc = self.L.oracle_count_ops(self.h, C.c_int(n), *self._src_args(src), first.ctypes.data_as(u64p),
                                     count.ctypes.data_as(u64p), C.c_int(int(early_reject)), _dp(out))
        if rc:
            raise RuntimeError("oracle_count_ops failed")
        keys = ("add", "mul", "div", "sqrt", "transcendental")
        return {"pre": dict(zip(keys, out[0:5])), "optics": dict(zip(keys, out[5:10])), "photons": int(out[10]),
                "survivors": float(out[11])}

    def trace_tangents(self, params, sources=None, first=None, count=None, n_threads=1):
        """Per-photon final positions and their derivatives with respect to each (surface, field) parameter."""
        src = self.scene.sources if sources is None else sources
        n = len(src)
        first = np.zeros(n, np.uint64) if first is None else _arr(first, np.uint64)
        count = _arr(src.n_photons if count is None else count, np.uint64)
        tot = int(count.sum())
        P = len(params)
        ps = _arr([p[0] for p in params], np.int32)
        pf = _arr([p[1] for p in params], np.int32)
        rx, ry = np.zeros(tot), np.zeros(tot)
        fl = np.zeros(tot, np.uint32)
        dx, dy = np.zeros((tot, P)), np.zeros((tot, P))
        u64p = C.POINTER(C.c_uint64)
        ip = C.POINTER(C.c_int)
        rc = self.L.oracle_trace_tangents(self.h, C.c_int(n), *self._src_args(src), first.ctypes.data_as(u64p),
                                          count.ctypes.data_as(u64p), C.c_int(P), ps.ctypes.data_as(ip),
                                          pf.ctypes.data_as(ip), _dp(rx), _dp(ry),
                                          fl.ctypes.data_as(C.POINTER(C.c_uint32)), _dp(dx), _dp(dy), C.c_int(n_threads))
        if rc:
            raise RuntimeError(f"oracle_trace_tangents failed ({rc})")
        return {"x": rx, "y": ry, "flags": fl, "dx": dx, "dy": dy, "source": np.repeat(np.arange(n), count.astype(np.int64))}


def philox(ctr, key):
    out = (C.c_uint32 * 4)()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    lib().oracle_philox(c, C.c_uint32(key[0]), C.c_uint32(key[1]), out)
    return [int(v) for v in out]


def zernike(j, rho, theta):
    rho = _arr(rho, np.float64); theta = _arr(theta, np.float64)
    out = np.zeros_like(rho)
    lib().oracle_zernike(C.c_int(j), C.c_int(len(rho)), _dp(rho), _dp(theta), _dp(out))
    return out


def film_reflectance(lam_nm, n0, n1, k1, t_mm, s):
    """Back-side reflection probability of the fringing calculation (single silicon layer, unpolarised)."""
    L = lib()
    L.oracle_film_reflectance.restype = C.c_double
    L.oracle_film_reflectance.argtypes = [C.c_double] * 6
    return L.oracle_film_reflectance(lam_nm, n0, n1, k1, t_mm, s)


def bleed(image, full_well):
    """Saturation and bleeding of a finished image (in place on a copy); returns (image, removed)."""
    img = np.ascontiguousarray(image, dtype=np.uint32).copy()
    L = lib()
    L.oracle_bleed.restype = C.c_uint64
    removed = L.oracle_bleed(img.ctypes.data_as(C.POINTER(C.c_uint32)), C.c_int(img.shape[1]), C.c_int(img.shape[0]),
                             C.c_uint32(int(full_well)))
    return img, int(removed)


def refract(d, N, n1, n2):
    out = np.zeros(3)
    rc = lib().oracle_refract(_dp(d), _dp(N), C.c_double(n1), C.c_double(n2), _dp(out))
    return rc, out


def reflect(d, N):
    out = np.zeros(3)
    lib().oracle_reflect(_dp(d), _dp(N), _dp(out))
    return out


def moments(rec, n_src):
    """Per-source detected count, centroid and central second moments (two-pass, FP64)."""
    out = np.zeros((n_src, 6))
    det = (rec["flags"] & F_DETECTED) != 0
    for s in range(n_src):
        m = det & (rec["source"] == s)
        x, y = rec["x"][m], rec["y"][m]
        if len(x) == 0:
            continue
        mx, my = x.mean(), y.mean()
        out[s] = [len(x), mx, my, ((x - mx) ** 2).mean(), ((x - mx) * (y - my)).mean(), ((y - my) ** 2).mean()]
    return out
