"""Sharding of the transport over ranks (one GPU per rank).

Packages are independent Philox streams indexed by their id, so rank r of W follows
ids [r n, (r+1) n) into its own absorption counts and escaped spectrum; the one
exchange is an exact integer sum of those arrays over ranks, after which every rank
can invert the summed counts into temperatures with eps = L_in / (n W). In the
frozen-temperature mode the sharded result equals the unsharded one exactly."""
from __future__ import annotations


def package_range(rank: int, world: int, n_per_rank: int):
    """(first id, count) of the packages rank `rank` follows."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("bad rank/world/n")
    return rank * n_per_rank, n_per_rank


def total_packages(world: int, n_per_rank: int) -> int:
    return world * n_per_rank


def sum_over_ranks(tensor, group=None):
    """In-place integer sum of a counts/spectrum tensor over all ranks."""
    import torch.distributed as dist
    dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
