"""The multi-GPU split on CPU: two gloo ranks trace disjoint photon ranges of the same stars with the oracle;
the sum of their images is the image of the whole range traced by one process, the job reduce (image, moment
sums, detected counts summed over the ranks) is consistent and equals the whole range's, and the timing
reduction is the maximum over ranks."""
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
    # the job's result as the benchmark forms it: image, moment sums and detected counts summed over the ranks
    import torch
    det = (rec["flags"] & 1) == 1
    mom = torch.zeros((1, 8), dtype=torch.float64)
    mom[0, 0] = float(det.sum())
    mom[0, 1] = float(rec["x"][det].sum())
    image = torch.as_tensor(rec["image"].astype(np.int32))
    job = sharding.reduce_job(image, mom, int(det.sum()))
    assert job["ranks"] == 2 and job["consistent"], job
    if rank == 0:
        np.save(out, np.r_[img.ravel(), t, job["detected"], mom[0, 1].item()])
    dist.destroy_process_group()


def test_two_ranks_sum_to_one_longer_exposure(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "img.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    res = np.load(out)
    img, t, det, sx = res[:-4], res[-4:-2], res[-2], res[-1]
    assert list(t) == [2.0, 0.0]
    from oracle import oracle
    from paper_1504_06570_gb300 import inputs as I
    sc = I.paraboloid_scene(n_photons=6000, screen_n=128)
    whole = oracle.Oracle(sc).trace(n_threads=1)
    ref = whole["image"].astype(np.int64).ravel()
    assert np.array_equal(img, ref)
    d = (whole["flags"] & 1) == 1
    assert det == d.sum() and abs(sx - whole["x"][d].sum()) < 1e-9 * max(1.0, abs(sx))
