"""The device Philox4x32-10 against the published known-answer vectors and against the oracle's independent
implementation on random counters and keys."""
import ctypes as C
import os

import numpy as np
import pytest

from paper_1504_06570_gb300 import phosim as P

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def device_philox(ctr, key):
    L = P.lib()
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint32)
    out = np.zeros_like(ctr)
    u32p = C.POINTER(C.c_uint32)
    assert L.phosim_philox(ctr.ctypes.data_as(u32p), key.ctypes.data_as(u32p), out.ctypes.data_as(u32p), len(ctr)) == 0
    return out


def test_known_answers():
    for line in open(GOLDEN):
        if not line.strip() or line[0] == "#":
            continue
        v = [int(x, 16) for x in line.split()]
        assert device_philox([v[0:4]], v[4:6])[0].tolist() == v[6:10]


def test_matches_oracle_on_random_counters(oracle_mod):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(512, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
    out = device_philox(ctr, key)
    for i in range(0, 512, 37):
        assert out[i].tolist() == oracle_mod.philox(ctr[i].tolist(), key.tolist())
