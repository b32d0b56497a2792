"""Sharding of the transport over ranks (one GPU per rank).

Packages are independent Philox streams indexed by their id, so rank r of W follows
ids [r n, (r+1) n) into its own absorption counts and escaped spectrum; the one
exchange is an exact integer sum of those arrays over ranks, after which every rank
inverts the summed counts into temperatures with eps = L_in / (n W). In the
frozen-temperature mode the sharded result equals the unsharded one exactly.

In the Bjorkman-Wood mode a rank only sees its own share of a cell's absorptions
while it transports. Its n-th absorption in a cell therefore indexes the temperature
at W n (``count_scale``): the rank's re-emission spectra then telescope to the
cell's total in expectation, as one process following all packages does; indexing
at n would re-emit every rank's share as if the cell held a W-th of its energy.
"""
from __future__ import annotations


def package_range(rank: int, world: int, n_per_rank: int):
    """(first id, count) of the packages rank `rank` follows."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("bad rank/world/n")
    return rank * n_per_rank, n_per_rank


def total_packages(world: int, n_per_rank: int) -> int:
    return world * n_per_rank


def count_scale(world: int) -> int:
    """Temperature-index scale of the BW re-emission when each of `world` ranks keeps
    its own counts (rt_run_opts.count_scale)."""
    if world < 1:
        raise ValueError("bad world size")
    return world


def sum_over_ranks(tensor, group=None):
    """In-place integer sum of a counts/spectrum tensor over all ranks."""
    import torch.distributed as dist
    dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


def reduce_counts(grid, buf, stream=None, group=None):
    """Make the grid's absorption counts the sum over all ranks: the library's counts
    into `buf` (int64 tensor [S][N]; on the device for NCCL, in host memory for gloo),
    the sum over ranks, and the sum back into the grid (rt_counts, all_reduce,
    rt_set_counts). Temperatures computed afterwards are those of all packages."""
    import torch
    grid.counts(out=buf, stream=stream)
    if buf.is_cuda:
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            sum_over_ranks(buf, group)
    else:  # a host copy has completed when rt_counts returns
        sum_over_ranks(buf, group)
    grid.set_counts(buf, stream=stream)
    return buf


def reduce_spectrum(grid, buf, stream=None, group=None):
    """The escaped spectrum [2][n_dir][B] summed over ranks into `buf` (int64)."""
    import torch
    grid.sed(out=buf, stream=stream)
    if buf.is_cuda:
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            sum_over_ranks(buf, group)
    else:
        sum_over_ranks(buf, group)
    return buf
