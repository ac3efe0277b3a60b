"""Pooling the steerable covariance over processes (one per GPU).

Images are independent (Sec. IV splits them over workers), so each rank
expands and accumulates its own shard; the only exchange is one all-gather
of the per-rank statistics [n, mean0, packed C] followed by the host-side
pooling of ffb_cov_merge.  torch.distributed carries the bytes (gloo or nccl);
the arithmetic is the library's.
"""
import numpy as np
import torch
import torch.distributed as dist

from .ffb import cov_merge


def pool_states(local_state, p, group=None):
    """All-gather float64 states of equal length and pool them; returns the
    pooled state (numpy) on every rank."""
    world = dist.get_world_size(group)
    t = torch.from_numpy(np.ascontiguousarray(local_state, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    states = np.stack([x.cpu().numpy() for x in parts])
    return cov_merge(p, states)


def pooled_covariance(plan, group=None):
    """Replace the plan's covariance by the pool over all ranks of ``group``."""
    pooled = pool_states(plan.cov_export(), plan.p, group)
    plan.cov_import(pooled)
    return pooled
