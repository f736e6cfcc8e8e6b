"""Work split across GPUs (one process per GPU).

Photons are independent given the counter-based streams, so N ranks trace disjoint photon ranges of the
same sources with no collective inside the trace: rank r takes photons [r n_s, (r + 1) n_s) of source s (weak
scaling: a longer exposure per GPU).  Images and moment sums are additive, so the job's result is one
sum-reduce (reduce_job), the path's only exchange step; timings are reduced by their maximum over ranks.
"""
from __future__ import annotations

import numpy as np


def rank_photon_range(counts, rank, world):
    """(first, count) per source for this rank under weak scaling."""
    counts = np.asarray(counts, np.uint64)
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return (counts * np.uint64(rank)).astype(np.uint64), counts.copy()


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_over_ranks(array, device=None):
    """Sum of an additive result (image, moment sums) over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(array), device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def reduce_job(image, moments, detected):
    """The job's result from every rank's part (photon ranges are disjoint): the image, the per-source moment sums
    and the detected count summed over the ranks, in place (torch tensors on the rank's device, or on the CPU
    with a gloo group).  Returns a summary whose 'consistent' is true when the job's image holds every rank's
    detected photons once and the moment sums count them once."""
    import torch
    import torch.distributed as dist
    det = torch.tensor([float(detected)], dtype=torch.float64, device=image.device)
    ranks = 1
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        ranks = dist.get_world_size()
        for t in (image, moments, det):
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = {"ranks": ranks, "detected": int(det.item()), "image_sum": int(image.to(torch.int64).sum().item()),
           "moment_count_sum": float(moments[:, 0].sum().item())}
    out["consistent"] = out["image_sum"] == out["detected"] and out["moment_count_sum"] == float(out["detected"])
    return out
