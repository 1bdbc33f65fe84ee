"""Multi-rank host logic on CPU (gloo, world size 2): two ranks with disjoint trajectory
blocks and one final exchange reproduce the single-process accumulator exactly -- the
summed ensemble spectra and, at their global trajectory indices, every trajectory's
diagnostics and winding records.  The per-rank work is done by the CPU oracle here; on
GPUs it is the library, which writes the same slot layout."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import gpe_oracle as O
from oracle.philox import tw_noise
from paper_2310_03636_gb300 import sharding

SHAPE, NLOCAL, SEED, DT = (16,), 2, 99, 0.05
STEPS = (3, 7)        # two sample slots


def accumulator(traj_ids):
    """Accumulator slots in the library's layout for the given global trajectories: per
    slot [4 nbins spectra | 8 diagnostics per trajectory | winding per trajectory]."""
    psis = []
    for t in traj_ids:
        e = tw_noise(SHAPE, SEED, t, 0.5, 1.0)
        e[1] += 1.0
        psis.append(e)
    p = torch.as_tensor(np.stack(psis))
    bins = O.radial_bins(SHAPE)
    slots = []
    done = 0
    for n in STEPS:
        p = O.propagate(p, DT, n - done, 1.0, -0.1, 0.09, 1.0, 1)
        done = n
        nk = O.bin_sum(O.occupation_modes(p, 1.0, 1), bins).sum(0)
        sk = O.bin_sum(O.spin_structure_modes(p, 1.0, 1), bins).sum(0)
        dg = O.diagnostics(p, 1.0, 1.0, -0.1, 0.09, 1)
        wn = O.winding_number(p)
        slots.append(torch.cat([nk.reshape(-1), sk.reshape(-1), dg.reshape(-1), wn.reshape(-1)]))
    return torch.cat(slots), int(bins.max()) + 1


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    base = sharding.trajectory_base(rank, NLOCAL)
    acc, nb = accumulator(range(base, base + NLOCAL))
    got = sharding.combine_accumulators(acc, len(STEPS), nb, NLOCAL, ws)
    torch.save(got, out + f".{rank}")
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_accumulator_equals_single_batch(tmp_path):
    out = str(tmp_path / "acc.pt")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    ref, nb = accumulator(range(2 * NLOCAL))
    sd = sharding.slot_doubles(nb, 2 * NLOCAL)
    assert ref.numel() == len(STEPS) * sd
    for r in range(2):
        got = torch.load(out + f".{r}")
        assert got.shape == ref.shape
        assert torch.allclose(got, ref, rtol=1e-13, atol=1e-12)
        # per-trajectory records are the single batch's, trajectory by trajectory
        g, f = got.reshape(len(STEPS), sd), ref.reshape(len(STEPS), sd)
        for t in range(2 * NLOCAL):
            o = 4 * nb + 8 * t
            assert torch.equal(g[:, o:o + 8], f[:, o:o + 8])
            w = 4 * nb + 8 * 2 * NLOCAL + t
            assert torch.equal(g[:, w], f[:, w])


def test_single_rank_and_bad_sizes():
    acc, nb = accumulator(range(NLOCAL))
    assert torch.equal(sharding.combine_accumulators(acc, len(STEPS), nb, NLOCAL, 1), acc)
    with pytest.raises(ValueError):
        sharding.combine_accumulators(acc[:-1], len(STEPS), nb, NLOCAL, 1)


def test_trajectory_blocks_are_disjoint():
    ranges = [set(range(sharding.trajectory_base(r, 64), sharding.trajectory_base(r, 64) + 64)) for r in range(8)]
    assert sum(len(r) for r in ranges) == len(set().union(*ranges)) == 512
