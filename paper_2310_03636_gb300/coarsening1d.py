"""Universal coarsening of the 1D spin-1 gas after a quench into the easy-plane phase
(Sec. 1, Figs. 1-2; Sec. 2.2 for the method): many truncated-Wigner trajectories start
from the polar state psi_0 = sqrt(n) with half a particle of noise per mode and evolve
with 0 < q < 2 n |c1| (c1 < 0).  The couplings are given as c0 n and c1 n, so that the
density n (atoms per lattice cell) sets only the relative size of the initial quantum
noise; it must be large (the default is 1000) for the noise to seed, rather than swamp,
the spin instability.  At logarithmically spaced times the library accumulates
the transverse spin structure factor S_perp(k, t), the diagnostics and the winding number
of the Larmor angle per trajectory; the host then fits the IR scaling exponents of
Eq. (StructureFactor) (scaling.py).  Every propagation step and every observable runs in
the library's kernels; this module only schedules the calls and fits on the host.

Usage: python -m paper_2310_03636_gb300.coarsening1d --ntraj 304 --t-end 40000 --out run.npz
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import binding as B
from . import scaling


def sample_steps(nsteps, nsamples, first):
    """Distinct step counts, logarithmically spaced from ``first`` to ``nsteps``."""
    s = np.unique(np.round(np.geomspace(max(1, first), nsteps, nsamples)).astype(np.int64))
    return [int(x) for x in s]


def run(n=4096, ntraj=304, dt=0.04, t_end=4.0e4, nsamples=20, t_first=200.0, c0n=1.0, c1n=-0.1, q=0.09,
        density=1000.0, seed=20231005, dtype="c64", chunk=2500, kmax_ir=0.15, t_fit=2000.0,
        uv_window=(0.3, 1.0), zeta_window=(0.05, 0.3)):
    c0, c1 = c0n / density, c1n / density
    nsteps = int(round(t_end / dt))
    steps = sample_steps(nsteps, nsamples, int(round(t_first / dt)))
    b = B.GPEBatch((n,), ntraj, dtype, c0, c1, q, dt)
    b.init_noise(seed, (0.0, 0.0, math.sqrt(density), 0.0, 0.0, 0.0), 0.5)
    nb, sd = b.layout()
    acc = b.new_accumulator(len(steps) + 1)
    flags = B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG | B.GPE_OBS_WINDING
    b.observables(acc, flags, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cur = 0
    for i, target in enumerate(steps):
        while cur < target:
            k = min(chunk, target - cur)
            b.step(k)
            cur += k
        b.observables(acc, flags, i + 1)
    st = b.sync_status()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if st != B.GPE_OK:
        raise B.GPEError(st, "device status after the run")
    counts = b.bin_counts().astype(np.float64)
    a = acc.cpu().numpy().reshape(len(steps) + 1, sd)
    times = np.array([0.0] + [s * dt for s in steps])
    S = np.empty((len(times), nb))
    nm = np.empty((len(times), 3, nb))
    N = np.empty((len(times), ntraj))
    Q = np.empty((len(times), ntraj))
    for j in range(len(times)):
        spec, diag = B.unpack_slot(a[j], nb, ntraj)
        S[j] = spec[3] / (counts * ntraj)
        nm[j] = spec[:3] / (counts * ntraj)
        N[j] = diag[:, :3].sum(1)
        Q[j] = B.unpack_winding(a[j], nb, ntraj)
    b.close()
    kbin = 2 * np.pi * np.arange(nb) / n
    late = times >= t_fit
    res = {"n": n, "ntraj": ntraj, "dt": dt, "t_end": nsteps * dt, "c0n": c0n, "c1n": c1n, "q": q, "density": density,
           "dtype": dtype, "steps": nsteps, "wall_s": wall,
           "site_updates_per_s": n * 3.0 * nsteps * ntraj / wall,
           "norm_drift": float(np.abs(N[-1] / N[0] - 1.0).max()),
           "winding_integer_dev": float(np.abs(Q - np.round(Q)).max()),
           "mean_abs_winding_last": float(np.abs(np.round(Q[-1])).mean()),
           "kmax_ir": kmax_ir, "t_fit": t_fit}
    if late.sum() >= 3:
        tl, Sl = times[late], S[late]
        a_m, b_m = scaling.moment_exponents(tl, kbin, Sl, kmax=kmax_ir)
        t_ref = float(tl[len(tl) // 2])
        a_c, b_c, r_c = scaling.collapse_exponents(tl, kbin, Sl, t_ref=t_ref, kmax=kmax_ir)
        res.update({"beta_moment": b_m, "alpha_moment": a_m, "beta_collapse": b_c, "alpha_collapse": a_c,
                    "collapse_residual": r_c, "t_ref": t_ref})
        # UV window (the paper's second scaling region) and the power-law fall-off k^-zeta
        a_u, b_u, r_u = scaling.collapse_exponents(tl, kbin, Sl, t_ref=t_ref, kmax=uv_window[1], kmin=uv_window[0],
                                                   guess=(-0.1, -0.1))
        zm = (kbin > zeta_window[0]) & (kbin < zeta_window[1])
        zeta = -scaling.fit_power(kbin[zm], S[-1][zm])[0]
        res.update({"uv_window": list(uv_window), "beta_uv": b_u, "alpha_uv": a_u, "uv_residual": r_u,
                    "zeta_window": list(zeta_window), "zeta": zeta})
    return res, {"times": times, "k": kbin, "S_perp": S, "n_m": nm, "N": N, "Q_w": Q, "counts": counts}


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--ntraj", type=int, default=304)
    p.add_argument("--dt", type=float, default=0.04)
    p.add_argument("--t-end", type=float, default=4.0e4)
    p.add_argument("--samples", type=int, default=20)
    p.add_argument("--t-first", type=float, default=200.0)
    p.add_argument("--q", type=float, default=0.09)
    p.add_argument("--c0n", type=float, default=1.0, help="c0 times the density")
    p.add_argument("--c1n", type=float, default=-0.1, help="c1 times the density")
    p.add_argument("--density", type=float, default=1000.0, help="atoms per lattice cell")
    p.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    p.add_argument("--kmax-ir", type=float, default=0.15)
    p.add_argument("--t-fit", type=float, default=2000.0)
    p.add_argument("--seed", type=int, default=20231005)
    p.add_argument("--out", default=None, help="write the spectra and windings to this .npz")
    a = p.parse_args()
    res, arrays = run(a.n, a.ntraj, a.dt, a.t_end, a.samples, a.t_first, a.c0n, a.c1n, a.q, a.density,
                      seed=a.seed, dtype=a.dtype, kmax_ir=a.kmax_ir, t_fit=a.t_fit)
    if a.out:
        np.savez_compressed(a.out, **arrays)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
