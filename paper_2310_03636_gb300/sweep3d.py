"""Quench sweep of the 3D spin-1 gas: the polar state psi_0 = sqrt(n) with half a particle of
noise per mode (Sec. 2.2) evolved at several quadratic Zeeman energies q across the
easy-plane window 0 < q < 2 n |c1| (c1 < 0), with the conserved quantities logged: the
total atom number N, the longitudinal magnetisation F_z = N_1 - N_-1 and the energy E of the
GPE functional, per trajectory, every ``sample_every`` steps.  The exact flow conserves all
three; the split step conserves N to rounding and E and F_z to O(dt^2), so their drifts are
the run's check of the integrator at this grid and step.  Every propagation step and every
diagnostic runs in the library's kernels; this module schedules the calls and summarises
the per-trajectory records on the host.

Usage: python -m paper_2310_03636_gb300.sweep3d --n 256 --ntraj 8 --steps 2000 --out sweep.json
"""
import argparse
import json
import time

import numpy as np


def drift_summary(diag):
    """diag: (samples, ntraj, 8) records (N_1, N_0, N_-1, E_kin, E_q, E_c0, E_c1, E_V) at the
    sample times, the first at t = 0.  Returns, per sample, the ensemble totals N, F_z, E
    and the largest per-trajectory drifts |N - N(0)| / N(0), |F_z - F_z(0)| / N(0) and
    |E - E(0)| / |E(0)|."""
    d = np.asarray(diag, dtype=np.float64)
    n = d[:, :, 0] + d[:, :, 1] + d[:, :, 2]
    fz = d[:, :, 0] - d[:, :, 2]
    e = d[:, :, 3:8].sum(axis=2)
    n0, fz0, e0 = n[0], fz[0], e[0]
    return {
        "N": n.sum(axis=1).tolist(),
        "F_z": fz.sum(axis=1).tolist(),
        "E": e.sum(axis=1).tolist(),
        "max_rel_dN": np.abs((n - n0) / n0).max(axis=1).tolist(),
        "max_rel_dFz": np.abs((fz - fz0) / n0).max(axis=1).tolist(),
        "max_rel_dE": np.abs((e - e0) / np.abs(e0)).max(axis=1).tolist(),
    }


def run_one(n, ntraj, q, steps, sample_every, dt=0.02, c0=1.0, c1=-0.1, seed=20231005, dtype="c64"):
    import torch

    from . import binding as B
    shape = (n, n, n)
    b = B.GPEBatch(shape, ntraj, dtype, c0, c1, q, dt)
    try:
        b.init_noise(seed, (0.0, 0.0, 1.0, 0.0, 0.0, 0.0), 0.5)
        nb, sd = b.layout()
        nsamples = steps // sample_every + 1
        acc = b.new_accumulator(nsamples)
        b.observables(acc, B.GPE_OBS_DIAG, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(1, nsamples):
            b.step(sample_every)
            b.observables(acc, B.GPE_OBS_DIAG, i)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = b.sync_status()
        if st != B.GPE_OK:
            raise B.GPEError(st, "device status after the run")
        a = acc.cpu().numpy().reshape(nsamples, sd)
        diag = np.stack([B.unpack_slot(a[i], nb, ntraj)[1] for i in range(nsamples)])
    finally:
        b.close()
    out = {"q": q, "steps": (nsamples - 1) * sample_every, "sample_every": sample_every,
           "t": [i * sample_every * dt for i in range(nsamples)], "wall_s": wall,
           "site_updates_per_s": n ** 3 * 3 * ntraj * (nsamples - 1) * sample_every / wall}
    out.update(drift_summary(diag))
    return out


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--ntraj", type=int, default=8)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--sample-every", type=int, default=100)
    p.add_argument("--q-factors", type=float, nargs="+", default=[0.3, 0.9, 1.5],
                   help="q in units of n |c1| (n = 1, c1 = -0.1)")
    p.add_argument("--dtype", default="c64")
    p.add_argument("--out", default=None)
    a = p.parse_args()
    runs = [run_one(a.n, a.ntraj, f * 0.1, a.steps, a.sample_every, dtype=a.dtype) for f in a.q_factors]
    res = {"grid": [a.n] * 3, "ntraj": a.ntraj, "dtype": a.dtype, "runs": runs}
    for r in runs:
        print(json.dumps({"q": r["q"], "steps": r["steps"], "wall_s": round(r["wall_s"], 3),
                          "site_updates_per_s": r["site_updates_per_s"], "max_rel_dN": max(r["max_rel_dN"]),
                          "max_rel_dFz": max(r["max_rel_dFz"]), "max_rel_dE": max(r["max_rel_dE"])}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
