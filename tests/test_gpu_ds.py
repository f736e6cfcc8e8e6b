"""The double-single primitives of the MIXED_DS path against FP64 on the host: each result within its error
bound (a few units of 2^-48, the double-single rounding level) of the exact FP64 value of the same
double-single inputs, the uniform draw exact, and the 2 pi u sine and cosine within 1e-14."""
import ctypes as C

import numpy as np
import pytest

from paper_1504_06570_gb300 import phosim as P

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def ds_round(v):
    """The value of the nearest double-single pair of v, as the device forms it."""
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


def ds_eval(op, a, b=None):
    L = P.lib()
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(a if b is None else b, np.float64)
    out = np.zeros(len(a) * (2 if op in (7, 9) else 1))
    dp = C.POINTER(C.c_double)
    rc = L.phosim_ds_eval(op, a.ctypes.data_as(dp), b.ctypes.data_as(dp), out.ctypes.data_as(dp), len(a))
    assert rc == 0
    return out


def operands(rng, n, lo=-6, hi=6, signed=True):
    v = 10.0 ** rng.uniform(lo, hi, n) * rng.uniform(1.0, 2.0, n)
    if signed:
        v *= rng.choice([-1.0, 1.0], n)
    return v


def test_arithmetic_error_bounds():
    rng = np.random.default_rng(1)
    n = 20000
    a, b = operands(rng, n), operands(rng, n)
    # near cancellation: b = -a (1 + tiny)
    b[:2000] = -a[:2000] * (1.0 + rng.uniform(-1e-9, 1e-9, 2000))
    A, B = ds_round(a), ds_round(b)
    u = 2.0 ** -48
    big = np.maximum(np.abs(A), np.abs(B))
    assert np.all(np.abs(ds_eval(0, a, b) - (A + B)) <= 4 * u * big)
    assert np.all(np.abs(ds_eval(1, a, b) - (A - B)) <= 4 * u * big)
    prod = A * B
    assert np.all(np.abs(ds_eval(2, a, b) - prod) <= 4 * u * np.abs(prod))
    q = A / B
    assert np.all(np.abs(ds_eval(3, a, b) - q) <= 16 * u * np.abs(q))
    f = prod + A
    assert np.all(np.abs(ds_eval(6, a, b) - f) <= 8 * u * np.maximum(np.abs(prod), np.abs(A)))


def test_roots_error_bounds():
    rng = np.random.default_rng(2)
    a = operands(rng, 20000, -12, 12, signed=False)
    a[:5] = [1.0, 4.0, 2.0, 1e-30, 1e30]
    A = ds_round(a)
    s = np.sqrt(A)
    assert np.all(np.abs(ds_eval(4, a) - s) <= 16 * 2.0 ** -48 * s)
    r = 1.0 / np.sqrt(A)
    assert np.all(np.abs(ds_eval(5, a) - r) <= 8 * 2.0 ** -48 * r)
    assert np.all(ds_eval(4, np.array([0.0, -1.0])) == 0.0)


def test_uniform_is_exact_and_sincos():
    rng = np.random.default_rng(3)
    w = np.concatenate([[0, 1, 255, 256, 2 ** 31, 2 ** 32 - 1, 2 ** 30, 3 * 2 ** 30, 2 ** 29],
                        rng.integers(0, 2 ** 32, 20000, dtype=np.uint64)]).astype(np.float64)
    u = (w + 0.5) * 2.0 ** -32
    assert np.array_equal(ds_eval(8, w), u)
    sc = ds_eval(7, w).reshape(-1, 2)
    assert np.abs(sc[:, 0] - np.sin(2 * np.pi * u)).max() < 1e-14
    assert np.abs(sc[:, 1] - np.cos(2 * np.pi * u)).max() < 1e-14
    assert np.abs(np.hypot(sc[:, 0], sc[:, 1]) - 1.0).max() < 1e-14


def test_floor_and_fraction():
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.uniform(-2e4, 2e4, 20000), [3.0, -3.0, 0.0, 1e4, 2.0 - 2.0 ** -40, -2.0 ** -40,
                                                        4097.0 + 2.0 ** -30, 4097.0 - 2.0 ** -30]])
    A = ds_round(a)
    ff = ds_eval(9, a).reshape(-1, 2)
    assert np.array_equal(ff[:, 0], np.floor(A))
    assert np.all((ff[:, 1] >= 0.0) & (ff[:, 1] <= 1.0))
    assert np.abs(ff[:, 1] - (A - np.floor(A))).max() < 1.5e-7
