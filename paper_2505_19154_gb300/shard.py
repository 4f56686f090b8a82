"""Sharding the path over views, one process per GPU.

Every (view, tile) unit of the rasterizer is independent, so views are
partitioned across ranks with no exchange while rendering.  Per-Gaussian
results are sums over views: the gradients of a multi-view step, and the
numerator and denominator of the feature fusion (Sec. 3.1,
f_g = sum_{v,p} w F / sum_{v,p} w).  Those are combined by one sum over ranks
before they are used; for fusion that is before the division, so the fused
feature on every rank equals the single-process result.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch


def view_shard(n_views: int, rank: int, world: int) -> range:
    """Contiguous block of views of `rank`; block sizes differ by at most one."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    base, extra = divmod(n_views, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def _world(group):
    dist = torch.distributed
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def allreduce_sum(tensors: Sequence[torch.Tensor], group=None) -> None:
    """In-place sum over ranks (nothing to do in a single process)."""
    if _world(group)[1] == 1:
        return
    for t in tensors:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM, group=group)


def fuse_sharded(rast, gaussians: tuple, views: Sequence[dict], maps_of: Callable[[int], torch.Tensor], D: int,
                 normalize: bool = False, group=None, dtype=torch.float32):
    """Feature fusion over all `views`, each rank taking its view_shard.

    `rast` provides fuse_accumulate(gaussians, views, maps, num, den) and
    fuse_finalize(gaussians, num, den, normalize) (api.Rasterizer does, on
    the GPU).  maps_of(v) returns view v's [H*W, D] float32 map; a rank asks
    only for its own views.  The library accumulates in float32; `dtype` is
    for other accumulators.  Returns (fused [N, D], num, den), the same on
    every rank."""
    rank, world = _world(group)
    means = gaussians[0]
    n = int(means.shape[0])
    num = torch.zeros((n, D), dtype=dtype, device=means.device)
    den = torch.zeros(n, dtype=dtype, device=means.device)
    for v in view_shard(len(views), rank, world):
        rast.fuse_accumulate(gaussians, [views[v]], [maps_of(v)], num, den)
    allreduce_sum([num, den], group)
    return rast.fuse_finalize(gaussians, num, den, normalize), num, den
