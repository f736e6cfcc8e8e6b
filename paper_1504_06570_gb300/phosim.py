"""Python binding of the phosim C ABI (include/phosim.h): argument marshalling only.

Every step of the photon path runs in the CUDA library libphosim.so; this module converts scenes from
`inputs` into the C structures, passes device pointers of torch tensors and the current CUDA stream, and
raises on error codes.  There is no CPU fallback: if the library is missing, importing `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as I

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libphosim.so")

MAX_SURFACES, MAX_LAYERS, MAX_SCALES, MAX_ZERNIKE = 16, 8, 2, 28
PLAIN_FP64, MIXED, MIXED_DS = 0, 1, 2
ATMOSPHERE, SENSOR, EARLY_REJECT, GRAPH, BACK_REFLECT, FRINGE = 1, 2, 4, 8, 16, 32
MOMENT_WORDS = 8
F_DETECTED = 1

STATUS = {0: "ok", -1: "invalid argument", -2: "out of device memory", -3: "CUDA error", -4: "unsupported",
          -5: "scene not ready", -6: "size exceeds a library maximum"}


class PhosimError(RuntimeError):
    def __init__(self, where, code):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


class SceneDesc(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("precision", C.c_int32), ("flags", C.c_uint32),
                ("pupil_r_in", C.c_double), ("pupil_r_out", C.c_double), ("h_top", C.c_double),
                ("z_entrance", C.c_double), ("lambda_ref", C.c_double), ("nx", C.c_int32), ("ny", C.c_int32),
                ("pixel", C.c_double), ("x0", C.c_double), ("y0", C.c_double), ("t_si", C.c_double),
                ("ell_lam0", C.c_double), ("ell_dlam", C.c_double), ("n_ell", C.c_int32),
                ("ell", C.POINTER(C.c_double)), ("n_sigma", C.c_int32), ("sigma", C.POINTER(C.c_double)),
                ("dead_layer", C.c_double), ("t_si_gx", C.c_double), ("t_si_gy", C.c_double)]


class Surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("material", C.c_int32), ("coating", C.c_int32), ("n_zern", C.c_int32),
                ("R", C.c_double), ("kappa", C.c_double), ("alpha", C.c_double * 8), ("z", C.c_double),
                ("r_in", C.c_double), ("r_out", C.c_double), ("pert", C.c_double * 6), ("zern_rnorm", C.c_double),
                ("zern", C.c_double * MAX_ZERNIKE)]


class Material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("B", C.c_double * 3), ("C", C.c_double * 3)]


class Coating(C.Structure):
    _fields_ = [("lam0", C.c_double), ("dlam", C.c_double), ("theta0", C.c_double), ("dtheta", C.c_double),
                ("n_lambda", C.c_int32), ("n_theta", C.c_int32), ("table", C.POINTER(C.c_double)),
                ("reflect", C.POINTER(C.c_double))]


class ScreenScale(C.Structure):
    _fields_ = [("pixel", C.c_double), ("n", C.c_int32), ("phase", C.POINTER(C.c_double))]


class Layer(C.Structure):
    _fields_ = [("z", C.c_double), ("vx", C.c_double), ("vy", C.c_double), ("n_scales", C.c_int32),
                ("scales", ScreenScale * MAX_SCALES)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("sed", C.c_int32), ("table", C.c_int32), ("bundle", C.c_int32),
                ("xi", C.c_double), ("eta", C.c_double), ("redshift", C.c_double), ("t0", C.c_double),
                ("t_exp", C.c_double), ("a", C.c_double), ("b", C.c_double), ("pa", C.c_double),
                ("bundle_sigma", C.c_double)]


RECORD_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("xc", "<f8"), ("yc", "<f8"), ("lam", "<f8"),
                         ("flags", "<u4"), ("pix", "<i4")])
assert RECORD_DTYPE.itemsize == 48

_lib = None

EXPORTS = ("phosim_create_scene", "phosim_load_optics", "phosim_load_screens", "phosim_load_seds",
           "phosim_load_sersic", "phosim_trace", "phosim_grad", "phosim_set_schedule", "phosim_get_counters",
           "phosim_destroy_scene", "phosim_status_string")


def lib():
    """The loaded CUDA library.  Raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libphosim.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.phosim_create_scene.argtypes = [C.POINTER(SceneDesc), C.POINTER(vp)]
        L.phosim_load_optics.argtypes = [vp, C.POINTER(Surface), C.c_int, C.POINTER(Material), C.c_int,
                                         C.POINTER(Coating), C.c_int]
        L.phosim_load_screens.argtypes = [vp, C.POINTER(Layer), C.c_int]
        L.phosim_load_seds.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double]
        L.phosim_load_sersic.argtypes = [vp, C.POINTER(C.c_double), C.c_int, C.c_int]
        L.phosim_trace.argtypes = [vp, C.POINTER(Source), C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                   vp, vp, vp, vp]
        L.phosim_grad.argtypes = [vp, C.POINTER(Source), C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), vp]
        L.phosim_set_schedule.argtypes = [vp, C.c_int, C.c_int]
        L.phosim_load_hf_kick.argtypes = [vp, C.POINTER(C.c_double), C.c_int]
        L.phosim_autotune.argtypes = [vp, C.POINTER(Source), C.c_int, C.POINTER(C.c_uint64), C.c_uint64, vp,
                                      C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.phosim_get_counters.argtypes = [vp, C.POINTER(C.c_uint64), C.c_int]
        L.phosim_get_schedule.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.phosim_moments_derive.argtypes = [C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double)]
        L.phosim_destroy_scene.argtypes = [vp]
        L.phosim_destroy_scene.restype = None
        L.phosim_status_string.argtypes = [C.c_int]
        L.phosim_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def _check(where, code):
    if code != 0:
        raise PhosimError(where, code)


def _dptr(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(C.POINTER(C.c_double))


def sources_struct(src: I.Sources):
    n = len(src)
    arr = (Source * max(n, 1))()
    for i in range(n):
        s = arr[i]
        s.kind = int(src.kind[i]); s.sed = int(src.sed[i]); s.table = int(src.table[i])
        s.xi = float(src.xi[i]); s.eta = float(src.eta[i]); s.redshift = float(src.redshift[i])
        s.t0 = float(src.t0[i]); s.t_exp = float(src.t_exp[i])
        s.a = float(src.a[i]); s.b = float(src.b[i]); s.pa = float(src.pa[i])
        if src.bundle is not None:
            s.bundle = int(src.bundle[i])
            s.bundle_sigma = float(src.bundle_sigma[i]) if src.bundle_sigma is not None else 0.0
    return arr


def surface_struct(s: I.Surface) -> Surface:
    d = Surface()
    d.kind, d.material, d.coating = int(s.kind), int(s.material), int(s.coating)
    d.R, d.kappa, d.z, d.r_in, d.r_out = float(s.R), float(s.kappa), float(s.z), float(s.r_in), float(min(s.r_out, 1e300))
    for i, a in enumerate(s.alpha):
        d.alpha[i] = float(a)
    for i, p in enumerate(s.pert):
        d.pert[i] = float(p)
    if len(s.zern) > MAX_ZERNIKE:
        raise ValueError("too many Zernike terms")
    d.n_zern = len(s.zern)
    d.zern_rnorm = float(s.zern_rnorm)
    for i, c in enumerate(s.zern):
        d.zern[i] = float(c)
    return d


class Scene:
    """A scene loaded into the CUDA library (device copies owned by the library)."""

    def __init__(self, scene: I.Scene, precision=PLAIN_FP64, early_reject=False, graph=False):
        L = lib()
        self.L = L
        self.scene = scene
        self.precision = precision
        d = scene.detector
        self._ell = np.ascontiguousarray(d.ell, np.float64)
        self._sig = np.ascontiguousarray(d.sigma, np.float64)
        desc = SceneDesc(seed=scene.seed, precision=precision,
                         flags=(ATMOSPHERE if scene.atmosphere else 0) | (SENSOR if scene.sensor else 0)
                         | (EARLY_REJECT if early_reject else 0) | (GRAPH if graph else 0)
                         | (BACK_REFLECT if getattr(scene, "back_reflect", False) else 0)
                         | (FRINGE if getattr(scene, "fringe", False) else 0),
                         pupil_r_in=scene.pupil_r_in, pupil_r_out=scene.pupil_r_out, h_top=scene.h_top,
                         z_entrance=scene.z_entrance, lambda_ref=scene.lambda_ref, nx=d.nx, ny=d.ny, pixel=d.pixel,
                         x0=d.x0, y0=d.y0, t_si=d.t_si, ell_lam0=d.ell_lam0, ell_dlam=d.ell_dlam,
                         n_ell=len(self._ell), ell=self._ell.ctypes.data_as(C.POINTER(C.c_double)),
                         n_sigma=len(self._sig), sigma=self._sig.ctypes.data_as(C.POINTER(C.c_double)),
                         dead_layer=float(getattr(d, "dead_layer", 0.0)), t_si_gx=float(getattr(d, "t_si_gx", 0.0)),
                         t_si_gy=float(getattr(d, "t_si_gy", 0.0)))
        h = C.c_void_p()
        _check("phosim_create_scene", L.phosim_create_scene(C.byref(desc), C.byref(h)))
        self.h = h
        self.load_optics(scene.surfaces, scene.materials, scene.coatings)
        self.load_screens(scene.layers if scene.atmosphere else [])
        flux = np.ascontiguousarray(scene.sed_flux, np.float64)
        _check("phosim_load_seds", L.phosim_load_seds(self.h, _dptr(flux), flux.shape[0], flux.shape[1],
                                                      scene.sed_lam0, scene.sed_dlam))
        sr = np.ascontiguousarray(scene.sersic, np.float64)
        _check("phosim_load_sersic", L.phosim_load_sersic(self.h, _dptr(sr), sr.shape[0], sr.shape[1]))
        hf = getattr(scene, "hf_kick", None)
        if hf is not None and len(hf):
            hq = np.ascontiguousarray(hf, np.float64)
            _check("phosim_load_hf_kick", L.phosim_load_hf_kick(self.h, _dptr(hq), len(hq)))
        self.src = None
        self.set_sources(scene.sources)

    def load_optics(self, surfaces, materials, coatings):
        n = len(surfaces)
        ss = (Surface * n)(*[surface_struct(s) for s in surfaces])
        ms = (Material * len(materials))()
        for i, m in enumerate(materials):
            ms[i].kind = m.kind
            for k in range(3):
                ms[i].B[k] = float(m.B[k]); ms[i].C[k] = float(m.C[k])
        keep = []
        cs = (Coating * max(1, len(coatings)))()
        for i, c in enumerate(coatings):
            T = np.ascontiguousarray(c.table, np.float64)
            keep.append(T)
            cs[i].lam0, cs[i].dlam, cs[i].theta0, cs[i].dtheta = c.lam0, c.dlam, c.theta0, c.dtheta
            cs[i].n_lambda, cs[i].n_theta = T.shape
            cs[i].table = T.ctypes.data_as(C.POINTER(C.c_double))
            if getattr(c, "reflect", None) is not None:
                Rf = np.ascontiguousarray(np.broadcast_to(c.reflect, T.shape), np.float64)
                keep.append(Rf)
                cs[i].reflect = Rf.ctypes.data_as(C.POINTER(C.c_double))
        _check("phosim_load_optics", self.L.phosim_load_optics(self.h, ss, n, ms, len(materials), cs, len(coatings)))

    def load_screens(self, layers):
        arr = (Layer * max(1, len(layers)))()
        keep = []
        for i, layer in enumerate(layers):
            arr[i].z, arr[i].vx, arr[i].vy = layer.z, layer.vx, layer.vy
            arr[i].n_scales = len(layer.scales)
            for q, sc in enumerate(layer.scales):
                ph = np.ascontiguousarray(sc.phase, np.float64)
                keep.append(ph)
                arr[i].scales[q].pixel = sc.pixel
                arr[i].scales[q].n = ph.shape[0]
                arr[i].scales[q].phase = ph.ctypes.data_as(C.POINTER(C.c_double))
        _check("phosim_load_screens", self.L.phosim_load_screens(self.h, arr, len(layers)))

    def set_sources(self, sources: I.Sources):
        self.sources = sources
        self.src = sources_struct(sources)
        self.n_photons = np.ascontiguousarray(sources.n_photons, np.uint64)

    def set_schedule(self, threads=0, tile=0):
        _check("phosim_set_schedule", self.L.phosim_set_schedule(self.h, int(threads), int(tile)))

    def trace(self, image, records=None, moments=None, n_photons=None, first=None, stream=None):
        """phosim_trace on torch tensors (image: int32 (ny, nx) on the device or on the host; records: uint8
        tensor of 48-byte records; moments: float64 (n_src, 8)).  Photon counts default to the sources'."""
        import torch
        n = len(self.sources)
        cnt = self.n_photons if n_photons is None else np.ascontiguousarray(n_photons, np.uint64)
        fst = None if first is None else np.ascontiguousarray(first, np.uint64)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        u64p = C.POINTER(C.c_uint64)
        _check("phosim_trace", self.L.phosim_trace(
            self.h, self.src, n, cnt.ctypes.data_as(u64p), None if fst is None else fst.ctypes.data_as(u64p),
            C.c_void_p(image.data_ptr()), None if records is None else C.c_void_p(records.data_ptr()),
            None if moments is None else C.c_void_p(moments.data_ptr()), C.c_void_p(stream) if stream else None))

    def grad(self, dL_dmoments, params, n_photons=None, stream=None):
        """phosim_grad: per-source gradients of sum_k dL[s, k] M_s[k], M = (mean x, mean y, Ixx, Ixy, Iyy),
        with respect to params = [(surface, field)] (field 0..5 = dx, dy, dz, tx, ty, tz; 100 + j = Zernike
        coefficient j + 1).  Returns (grad (n_src, n_params), moments (n_src, 6))."""
        import torch
        n = len(self.sources)
        cnt = self.n_photons if n_photons is None else np.ascontiguousarray(n_photons, np.uint64)
        dL = np.ascontiguousarray(dL_dmoments, np.float64).reshape(n, 5)
        ps = np.ascontiguousarray([int(p[0]) for p in params], np.int32)
        pf = np.ascontiguousarray([int(p[1]) for p in params], np.int32)
        g = np.zeros((n, len(params)))
        m = np.zeros((n, 6))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        i32p = C.POINTER(C.c_int32)
        _check("phosim_grad", self.L.phosim_grad(self.h, self.src, n, cnt.ctypes.data_as(C.POINTER(C.c_uint64)),
                                                 _dptr(dL), ps.ctypes.data_as(i32p), pf.ctypes.data_as(i32p),
                                                 len(params), g.ctypes.data_as(C.POINTER(C.c_double)),
                                                 m.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream)))
        return g, m

    def set_parameters(self, params, values):
        """Write surface misalignments / Zernike coefficients (same (surface, field) convention) into the
        scene's optics and reload them."""
        for (si, f), v in zip(params, np.asarray(values, np.float64)):
            s = self.scene.surfaces[si]
            if f < 6:
                pert = list(s.pert) + [0.0] * (6 - len(s.pert))
                pert[f] = float(v)
                s.pert = tuple(pert)
            else:
                j = f - 100
                z = list(s.zern) + [0.0] * max(0, j + 1 - len(s.zern))
                z[j] = float(v)
                s.zern = tuple(z)
        self.load_optics(self.scene.surfaces, self.scene.materials, self.scene.coatings)

    def autotune(self, sample_photons=5_000_000, n_photons=None, stream=None):
        """phosim_autotune on this scene's sources; returns (threads per block, photons per tile)."""
        import torch
        cnt = self.n_photons if n_photons is None else np.ascontiguousarray(n_photons, np.uint64)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        t, k = C.c_int(), C.c_int()
        _check("phosim_autotune", self.L.phosim_autotune(self.h, self.src, len(self.sources),
                                                         cnt.ctypes.data_as(C.POINTER(C.c_uint64)),
                                                         C.c_uint64(int(sample_photons)), C.c_void_p(stream),
                                                         C.byref(t), C.byref(k)))
        return t.value, k.value

    def schedule(self):
        """phosim_get_schedule: (threads per block, photons per warp tile) of the scene's trace launch."""
        t, k = C.c_int(), C.c_int()
        _check("phosim_get_schedule", self.L.phosim_get_schedule(self.h, C.byref(t), C.byref(k)))
        return t.value, k.value

    def counters(self):
        out = (C.c_uint64 * 10)()
        _check("phosim_get_counters", self.L.phosim_get_counters(self.h, out, 10))
        return np.array(out[:], np.uint64)

    def close(self):
        if getattr(self, "h", None):
            self.L.phosim_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bleed(image, full_well, stream=None):
    """phosim_bleed on a device int32 image tensor (in place); returns the number of removed electrons."""
    import torch
    removed = torch.zeros(1, dtype=torch.int64, device=image.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    L = lib()
    L.phosim_bleed.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint32, C.c_void_p, C.c_void_p]
    _check("phosim_bleed", L.phosim_bleed(C.c_void_p(image.data_ptr()), image.shape[1], image.shape[0],
                                          C.c_uint32(int(full_well)), C.c_void_p(removed.data_ptr()), C.c_void_p(stream)))
    return removed


def records_to_numpy(rec_tensor):
    return rec_tensor.cpu().numpy().view(RECORD_DTYPE)


def derived_moments(m):
    """(count, mean x, mean y, Ixx, Ixy, Iyy) per source from the additive sums of phosim_trace, by
    phosim_moments_derive (NaN for a source with no detected photon)."""
    if hasattr(m, "detach"):
        m = m.detach().cpu().numpy()
    m = np.ascontiguousarray(np.asarray(m, np.float64).reshape(-1, MOMENT_WORDS))
    out = np.zeros((m.shape[0], 6))
    dp = C.POINTER(C.c_double)
    _check("phosim_moments_derive", lib().phosim_moments_derive(m.ctypes.data_as(dp), m.shape[0], out.ctypes.data_as(dp)))
    return out


def _autograd_function():
    import torch

    class PSFMoments(torch.autograd.Function):
        """Per-source PSF moments (mean x, mean y, Ixx, Ixy, Iyy) as a differentiable function of surface
        parameters; the backward pass is the adjoint raytrace (phosim_grad) with common random numbers and
        the forward pass's accept decisions."""

        @staticmethod
        def forward(ctx, theta, scene, params):
            # one FP64 trace with per-source moment sums (the adjoint runs only in backward)
            scene.set_parameters(params, theta.detach().cpu().numpy())
            n = len(scene.sources)
            dev = torch.device("cuda", torch.cuda.current_device())
            d = scene.scene.detector
            img = torch.zeros((d.ny, d.nx), dtype=torch.int32, device=dev)
            sums = torch.zeros((n, MOMENT_WORDS), dtype=torch.float64, device=dev)
            if scene.precision != PLAIN_FP64:
                raise ValueError("PSFMoments needs a PLAIN_FP64 scene (the adjoint differentiates the FP64 path)")
            scene.trace(img, None, sums)
            m = derived_moments(sums)
            ctx.scene, ctx.params = scene, params
            return torch.as_tensor(np.nan_to_num(m[:, 1:]), dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, g):
            grad, _ = ctx.scene.grad(g.detach().cpu().numpy(), ctx.params)
            return torch.as_tensor(grad.sum(0), dtype=g.dtype, device=g.device), None, None

    return PSFMoments


def psf_moments(theta, scene, params):
    """Differentiable per-source PSF moments; see PSFMoments."""
    return _autograd_function().apply(theta, scene, params)
