"""Trajectory sharding across ranks (one process per GPU).

Trajectories are independent (the paper runs many of them per GPU and spreads ensembles
over several GPUs, Sec. 2.2), so N ranks each advance their own block of trajectories with
no exchange during propagation.  Rank r holds global trajectories
[r * n_local, (r + 1) * n_local) and draws their noise with the same seed (the global
index enters the Philox counter through gpe_batch_set_traj_base), so the N-rank ensemble is
exactly the single-batch ensemble of N * n_local trajectories.

The only exchange is the combination of the FP64 observable accumulators, once, at the end.
One accumulator slot of a batch of n trajectories (observables_accumulate) is

    [4 * nbins spectra | 8 * n diagnostics records | n winding numbers]

The spectra are sums over the batch's trajectories, so they add across ranks; the
diagnostics and winding records belong to single trajectories, so they are gathered and
placed at the rank's global trajectory offset.  The result has the layout one batch of
N * n_local trajectories would have written.
"""
import torch
import torch.distributed as dist


def trajectory_base(rank, n_local):
    """Global index of the rank's first trajectory."""
    return rank * n_local


def slot_doubles(nbins, ntraj):
    """Length of one accumulator slot for a batch of ``ntraj`` trajectories."""
    return 4 * max(nbins, 0) + 9 * ntraj


def combine_accumulators(acc, nslots, nbins, n_local, world_size):
    """Combines the ranks' accumulators into the single-batch layout of world_size * n_local
    trajectories: spectra summed over ranks (all-reduce), per-trajectory records gathered
    (all-gather) and placed at the global trajectory index.  ``acc``: this rank's
    accumulator, ``nslots`` slots of slot_doubles(nbins, n_local) doubles.  Every rank gets
    the combined accumulator (a new tensor; ``acc`` is not modified).  With one rank it
    returns a copy of ``acc``."""
    nb = max(nbins, 0)
    sd = slot_doubles(nbins, n_local)
    if acc.numel() != nslots * sd:
        raise ValueError(f"accumulator has {acc.numel()} doubles, expected {nslots} slots of {sd}")
    a = acc.reshape(nslots, sd)
    if world_size == 1:
        return acc.clone()
    spec = a[:, :4 * nb].contiguous()
    rec = a[:, 4 * nb:].contiguous()                 # (nslots, 9 n_local): diagnostics, then windings
    dist.all_reduce(spec, op=dist.ReduceOp.SUM)
    parts = [torch.empty_like(rec) for _ in range(world_size)]
    dist.all_gather(parts, rec)
    n_glob = world_size * n_local
    out = torch.empty((nslots, slot_doubles(nbins, n_glob)), dtype=acc.dtype, device=acc.device)
    out[:, :4 * nb] = spec
    diag = out[:, 4 * nb:4 * nb + 8 * n_glob]
    wind = out[:, 4 * nb + 8 * n_glob:]
    for r, p in enumerate(parts):
        base = trajectory_base(r, n_local)
        diag[:, 8 * base:8 * (base + n_local)] = p[:, :8 * n_local]
        wind[:, base:base + n_local] = p[:, 8 * n_local:]
    return out.reshape(-1)
