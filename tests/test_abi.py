"""The C ABI without a GPU: the library loads, exports what include/phosim.h declares, its structures have
the layout the binding assumes, and argument validation answers before any device work."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_1504_06570_gb300 import build as B
from paper_1504_06570_gb300 import phosim as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


@pytest.fixture(scope="module")
def L():
    B.build()
    return P.lib()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(phosim_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert {"phosim_create_scene", "phosim_load_optics", "phosim_load_screens", "phosim_trace", "phosim_grad"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (phosim_\w+)", out))
    assert names <= exported, names - exported
    for n in names:
        getattr(L, n)


def test_struct_layout_matches_header():
    """sizeof / offsetof of every ABI structure, compiled from the header with the system C compiler."""
    checks = {"phosim_scene_desc": (P.SceneDesc, ["seed", "precision", "ell", "n_sigma", "sigma", "dead_layer", "t_si_gy"]),
              "phosim_surface": (P.Surface, ["R", "alpha", "pert", "zern_rnorm", "zern"]),
              "phosim_material": (P.Material, ["B", "C"]),
              "phosim_coating": (P.Coating, ["n_lambda", "table", "reflect"]),
              "phosim_screen_scale": (P.ScreenScale, ["n", "phase"]),
              "phosim_layer": (P.Layer, ["n_scales", "scales"]),
              "phosim_source": (P.Source, ["bundle", "xi", "pa", "bundle_sigma"])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "phosim.h"', "int main(void){"]
    for st, (_, fields) in checks.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append('printf("phosim_photon_record %zu\\n", sizeof(phosim_photon_record));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "abi.c")
        exe = os.path.join(d, "abi")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = dict(l.rsplit(" ", 1) for l in subprocess.run([exe], capture_output=True, text=True).stdout.split("\n") if l)
    for st, (cls, fields) in checks.items():
        assert int(out[st]) == C.sizeof(cls), st
        for f in fields:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
    assert int(out["phosim_photon_record"]) == P.RECORD_DTYPE.itemsize


def test_argument_validation_before_device_work(L):
    h = C.c_void_p()
    assert L.phosim_create_scene(None, C.byref(h)) == -1
    desc = P.SceneDesc(precision=7, nx=16, ny=16, pixel=0.01, t_si=0.1, lambda_ref=500.0, ell_dlam=1.0)
    assert L.phosim_create_scene(C.byref(desc), C.byref(h)) == -1         # unknown precision
    desc.precision = 0
    desc.n_ell = 1                                                          # too short a table
    assert L.phosim_create_scene(C.byref(desc), C.byref(h)) == -1
    assert L.phosim_trace(None, None, 0, None, None, None, None, None, None) == -1
    assert L.phosim_load_optics(None, None, 0, None, 0, None, 0) == -1
    assert L.phosim_set_schedule(None, 64, 0) == -1
    assert L.phosim_status_string(-6) == b"size exceeds a library maximum"
    L.phosim_destroy_scene(None)


def test_probe_arguments_checked_before_device_work(L):
    """The measurement probes of phosim_bench.h reject their malformed arguments before any CUDA call, so these
    answers need no device."""
    r = C.c_double()
    assert L.phosim_fma_rate(0, 0, 4, None, C.byref(r)) == -1               # iterations < 1
    assert L.phosim_fma_rate(0, 10, 4, None, None) == -1                    # no output
    assert L.phosim_ds_rate(5, 10, 4, None, C.byref(r)) == -1               # unknown primitive
    assert L.phosim_ds_rate(-1, 10, 4, None, C.byref(r)) == -1
    assert L.phosim_ds_rate(0, 10, 0, None, C.byref(r)) == -1               # blocks per SM < 1
    for nbytes in (0, 32 * 1023, (1 << 20) + 16, 128 << 30):               # too small, not a multiple of 32, too large
        assert L.phosim_gather_rate(C.c_size_t(nbytes), 16, 4, None, C.byref(r)) == -1, nbytes
    assert L.phosim_gather_rate(C.c_size_t(1 << 20), 0, 4, None, C.byref(r)) == -1
    assert L.phosim_gather_rate(C.c_size_t(1 << 20), 16, 4, None, None) == -1
    assert L.phosim_moments_derive(None, 1, None) == -1
    assert L.phosim_ds_eval(10, None, None, None, 1) == -1


def test_moments_derive_on_the_host(L):
    """phosim_moments_derive is host arithmetic (Sec. 3.1 counts and centroids, the second moments of the
    image-quality comparisons): from sums about a reference point it gives the count, the centroid and the
    central second moments of a point set, computed here two-pass from the points themselves; NaN for a
    source with no photon."""
    import numpy as np
    rng = np.random.default_rng(5)
    pts = [rng.normal([3.0, -2.0], [0.02, 0.05], size=(n, 2)) for n in (1, 7, 1000)]
    sums = np.zeros((4, P.MOMENT_WORDS))
    for s, p in enumerate(pts):
        ref = np.array([2.99, -2.01])
        d = p - ref
        sums[s, :6] = [len(p), d[:, 0].sum(), d[:, 1].sum(), (d[:, 0] ** 2).sum(), (d[:, 0] * d[:, 1]).sum(),
                       (d[:, 1] ** 2).sum()]
        sums[s, 6:8] = ref
    out = P.derived_moments(sums)
    for s, p in enumerate(pts):
        c = p.mean(axis=0)
        q = p - c
        want = [len(p), c[0], c[1], (q[:, 0] ** 2).mean(), (q[:, 0] * q[:, 1]).mean(), (q[:, 1] ** 2).mean()]
        np.testing.assert_allclose(out[s], want, rtol=1e-9, atol=1e-13)
    assert np.all(np.isnan(out[3, 1:]))
    assert out[3, 0] == 0
