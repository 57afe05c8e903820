"""Trajectory sharding across ranks (one process per GPU).

Trajectories are independent (Sec. III.B repeats the procedure), and every draw is
keyed by the global trajectory index, so a run split over G ranks gives the
same per-trajectory results as one rank.  The only exchange is a host-side
gather of each rank's small result arrays; nothing crosses between GPUs on the
data path.
"""
import numpy as np


def shard_range(first, n, rank, world):
    """Contiguous share [lo, hi) of trajectories first..first+n-1 for this rank."""
    lo = first + (n * rank) // world
    hi = first + (n * (rank + 1)) // world
    return lo, hi


def interleaved_index(step, n_points, rank, world):
    """Trajectory index of a benchmark step that cycles over n_points noise points."""
    return (step // n_points) * world + rank


def run_sharded(run_fn, first, n, rank, world, group=None):
    """Run this rank's share with run_fn(lo, count) -> tuple of arrays (leading axis = trajectory),
    gather every rank's share (host-side, torch.distributed object gather) and return the
    concatenation in trajectory order on every rank."""
    lo, hi = shard_range(first, n, rank, world)
    local = run_fn(lo, hi - lo)
    if world == 1:
        return local
    import torch.distributed as dist

    parts = [None] * world
    dist.all_gather_object(parts, [np.asarray(a) for a in local], group=group)
    return tuple(np.concatenate([p[i] for p in parts], axis=0) for i in range(len(local)))
