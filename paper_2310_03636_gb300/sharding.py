"""Trajectory sharding across ranks (one process per GPU).

Trajectories are independent, so N ranks each advance their own block of trajectories
with no exchange during propagation.  Rank r holds global trajectories
[r * n_local, (r + 1) * n_local) and draws their noise with the same seed, so the N-rank
ensemble is exactly the single-batch ensemble of N * n_local trajectories.  The only
exchange is the sum of the FP64 observable accumulators, once, at the end.
"""
import torch
import torch.distributed as dist


def trajectory_base(rank, n_local):
    """Global index of the rank's first trajectory."""
    return rank * n_local


def reduce_accumulators(acc, world_size):
    """Sum the FP64 accumulators of all ranks in place (the ensemble exchange step).
    Per-trajectory diagnostics occupy disjoint slots only if each rank wrote its records
    at its global offset; spectra sums add up directly."""
    if world_size > 1:
        dist.all_reduce(acc, op=dist.ReduceOp.SUM)
    return acc
