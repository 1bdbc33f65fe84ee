"""Multi-rank host logic on CPU (gloo, world size 2): two ranks with disjoint trajectory
blocks and one final all-reduce reproduce the single-process ensemble spectra exactly
(the per-rank work is done by the CPU oracle here; on GPUs it is the library)."""
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

SHAPE, NLOCAL, SEED, DT, STEPS = (16, 16), 2, 99, 0.05, 4


def ensemble_spectra(traj_ids):
    psis = []
    for t in traj_ids:
        e = tw_noise(SHAPE, SEED, t, 0.5, 1.0)
        e[1] += 1.0
        psis.append(e)
    p = O.propagate(torch.as_tensor(np.stack(psis)), DT, STEPS, 1.0, -0.1, 0.09, 1.0, 2)
    bins = O.radial_bins(SHAPE)
    nk = O.bin_sum(O.occupation_modes(p, 1.0, 2), bins).sum(0)
    sk = O.bin_sum(O.spin_structure_modes(p, 1.0, 2), bins).sum(0)
    return torch.cat([nk.reshape(-1), sk.reshape(-1)])


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    base = sharding.trajectory_base(rank, NLOCAL)
    acc = ensemble_spectra(range(base, base + NLOCAL))
    sharding.reduce_accumulators(acc, ws)
    if rank == 0:
        torch.save(acc, out)
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_ensemble_equals_single_batch(tmp_path):
    out = str(tmp_path / "acc.pt")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = torch.load(out)
    ref = ensemble_spectra(range(2 * NLOCAL))
    assert torch.allclose(got, ref, rtol=1e-13, atol=1e-12)


def test_trajectory_blocks_are_disjoint():
    ranges = [set(range(sharding.trajectory_base(r, 64), sharding.trajectory_base(r, 64) + 64)) for r in range(8)]
    assert sum(len(r) for r in ranges) == len(set().union(*ranges)) == 512
