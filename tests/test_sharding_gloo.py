"""The multi-GPU split on CPU: two gloo ranks trace disjoint photon ranges of the same stars with the oracle;
the sum of their images is the image of the whole range traced by one process, and the timing reduction is
the maximum over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle
    from paper_1504_06570_gb300 import inputs as I
    from paper_1504_06570_gb300 import sharding
    sc = I.paraboloid_scene(n_photons=3000, screen_n=128)
    first, count = sharding.rank_photon_range(sc.sources.n_photons, rank, world)
    rec = oracle.Oracle(sc).trace(first=first, count=count, n_threads=1)
    img = sharding.sum_over_ranks(rec["image"].astype(np.int64))
    t = sharding.max_over_ranks([float(rank + 1), -float(rank)])
    if rank == 0:
        np.save(out, np.r_[img.ravel(), t])
    dist.destroy_process_group()


def test_two_ranks_sum_to_one_longer_exposure(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "img.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    res = np.load(out)
    img, t = res[:-2], res[-2:]
    assert list(t) == [2.0, 0.0]
    from oracle import oracle
    from paper_1504_06570_gb300 import inputs as I
    sc = I.paraboloid_scene(n_photons=6000, screen_n=128)
    ref = oracle.Oracle(sc).trace(n_threads=1)["image"].astype(np.int64).ravel()
    assert np.array_equal(img, ref)
