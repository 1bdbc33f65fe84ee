#!/usr/bin/env python
"""Throughput of the spin-1 GPE split-step hot path (site-updates/s).

Workload: 2D 512^2 periodic grid, 64 truncated-Wigner trajectories per GPU, complex64
fields with FP64 reductions, polar-state quench (c0 = 1, c1 = -0.1, q = 0.09), dt = 0.02,
ensemble spectra n_m(k) and S_perp(k) plus diagnostics every 250 steps.  One bench step
= one sampling interval: 250 time steps of the whole batch + one observables_accumulate.
site-updates = points x 3 components x time steps x trajectories.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run, one rank per GPU; trajectories are sharded
(each rank advances its own 64), the FP64 accumulators are combined across ranks once at
the end (spectra summed, per-trajectory records gathered: the path's only exchange step).
Rank 0 prints one JSON line.  Besides the K-step totals, every bench step is bracketed by
its own CUDA events, and the line reports the median and spread of those per-step times.
"""
import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2310_03636_gb300 import workloads as W  # noqa: E402

STEPS_PER_SAMPLE = 250
WL = W.C2_2D


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the ragged-batch measurement the default run adds under 'secondary'")
    p.add_argument("--workload", choices=["2d", "1d", "3d", "ragged", "adjoint", "paper1d", "paper1d_f64"], default="2d",
                   help="2d: the benchmark workload (default); others print a line for that configuration")
    p.add_argument("--no-autotune", action="store_true",
                   help="fixed default column-pass tile widths (for launch lists under ncu, whose timing "
                        "would mislead the tuner)")
    p.add_argument("--alu-peaks", action="store_true",
                   help="measure the FP32 / packed FP32 / FP64 FMA rates (roofline of the compute-bound passes)")
    p.add_argument("--ncu-case", action="store_true",
                   help="small profiling target: the 512^2 x 64 batch (403 MB > L2), 4 steps + observables")
    return p.parse_args()


def dist_setup(n):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarise(lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, maximum clock and the throttle reasons seen in nvidia-smi CSV
        lines of the query ``Q`` (no header, no units)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# Sources that define the propagation passes (x pass and strided passes); the ncu traffic
# figures in profiles/ stay valid while these are unchanged.
PASS_SOURCES = ("common.cuh", "fft.cuh", "local_step.cuh", "async_copy.cuh", "prop_kernels.cuh", "prop_f32.cu",
                "prop_f64.cu", "colpass_tma_f32.cu", "xpass_f32_small.cu", "xpass_f32_large.cu", "internal.h")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in PASS_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2310_03636_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class):
    """DRAM bytes per launch from the committed ncu summary, if the kernels are unchanged."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    v = d.get("per_launch_bytes", {}).get(kernel_class)
    return float(v) if v is not None else None


# ------------------------------------------------------------------ CPU oracle timing

def cpu_model():
    """Host CPU as /proc/cpuinfo names it (model name, or Arm implementer/part), and nproc."""
    name = None
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model"):
            for line in info:
                if line.lower().startswith(key.lower()):
                    name = line.split(":", 1)[1].strip()
                    break
            if name:
                break
        if not name:
            impl = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")), None)
            part = next((l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")), None)
            if impl or part:
                name = f"arm implementer {impl} part {part}"
    except OSError:
        pass
    return {"model": name or "unknown", "nproc": os.cpu_count()}


def oracle_sample(seconds_target=12.0):
    """Time the FP64 CPU oracle on a bounded sample of the workload: one 512^2 trajectory,
    as many Strang steps as fit in about ``seconds_target`` seconds, plus its spectra."""
    from oracle import gpe_oracle as O
    from oracle.philox import tw_noise
    psi = tw_noise(WL.shape, W.SEED_BASE, 0, WL.noise_per_mode, WL.dx)
    psi[1] += math.sqrt(WL.n)
    p = torch.as_tensor(psi)
    t0 = time.perf_counter()
    p = O.strang_step(p, WL.dt, WL.c0, WL.c1, WL.q, WL.dx, 2)
    one = time.perf_counter() - t0
    nsteps = max(1, int(seconds_target / max(one, 1e-3)))
    t0 = time.perf_counter()
    p = O.propagate(p, WL.dt, nsteps, WL.c0, WL.c1, WL.q, WL.dx, 2)
    bins = O.radial_bins(WL.shape)
    O.bin_sum(O.occupation_modes(p, WL.dx, 2), bins)
    O.bin_sum(O.spin_structure_modes(p, WL.dx, 2), bins)
    el = time.perf_counter() - t0
    su = WL.sites * 3 * nsteps
    return {"value": su / el, "unit": "site-updates/s", "cores": torch.get_num_threads(), "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"1 trajectory of the 512^2 workload, {nsteps} steps + one spectra evaluation, "
                      f"{el:.1f} s, FP64 torch CPU"}


def step_stats(ms_list):
    """Median and spread of per-bench-step times (ms) from CUDA events."""
    v = sorted(ms_list)
    n = len(v)
    if n == 0:
        return None
    q = lambda f: v[min(n - 1, max(0, int(round(f * (n - 1)))))]
    med = statistics.median(v)
    return {"n": n, "median_ms": med, "min_ms": v[0], "max_ms": v[-1], "p10_ms": q(0.1), "p90_ms": q(0.9),
            "spread_pct": 100.0 * (v[-1] - v[0]) / med if med > 0 else None}


def workload_config(ws):
    """The bench workload as both arms name it in their JSON line."""
    return {"workload": WL.name, "grid": list(WL.shape), "ntraj_per_gpu": WL.ntraj,
            "dt": WL.dt, "steps_per_bench_step": STEPS_PER_SAMPLE,
            "observables_every": STEPS_PER_SAMPLE, "c0": WL.c0, "c1": WL.c1, "q": WL.q,
            "parallelism": f"trajectories sharded over {ws} GPU(s)",
            "l2": "inputs larger than L2 (403 MB of fields per GPU)"}


def run_reference(args):
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    per_step = max(2.0, 40.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(per_step)
    vals = []
    t0 = time.perf_counter()
    samples = []
    for _ in range(args.steps):
        r = oracle_sample(per_step)
        vals.append(r["value"])
        samples.append(r["sample"])
    el = time.perf_counter() - t0
    value = float(np.mean(vals))
    out = {"impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(ws),
           "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": torch.get_num_threads(), "cpu": cpu_model(),
                            "kind": "oracle", "sample": samples[0] if samples else ""},
           "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    from paper_2310_03636_gb300 import binding as B
    ws, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    from paper_2310_03636_gb300 import sharding
    seed = W.SEED_BASE
    b = B.GPEBatch(WL.shape, WL.ntraj, "c64", WL.c0, WL.c1, WL.q, WL.dt, dx=WL.dx)
    b.set_traj_base(sharding.trajectory_base(rank, WL.ntraj))
    if args.no_autotune:
        b.set_autotune(False)
    nb, sd = b.layout()
    nslots = args.warmup + 2 * args.steps      # warm-up, timed and profiled samples
    acc = torch.zeros(nslots * sd, dtype=torch.float64, device=dev)
    b.init_noise(seed, WL.mean_spinor(), WL.noise_per_mode)
    for k in range(args.warmup):
        b.step(STEPS_PER_SAMPLE)
        b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, k)
    torch.cuda.synchronize()
    assert b.sync_status() == B.GPE_OK

    clocks = Clocks(dev.index)
    su_per_step = WL.site_updates_per_step * STEPS_PER_SAMPLE
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    l0 = B.gpe_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(stream)
    ev[0].record(stream)
    for k in range(args.steps):
        b.step(STEPS_PER_SAMPLE)
        b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, args.warmup + k)
        ev[k + 1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = B.gpe_launch_count() - l0
    per_step = step_stats([ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)])
    barrier(ws)
    # Per-kernel times for the roofline: the same K bench steps once more, each launch
    # bracketed by CUDA events on its stream (kept out of the region above, where the
    # ~5000 event records per run would add about 1 % of gaps between kernels).
    B.gpe_profile_enable(b.h, True)
    B.gpe_profile_read(b.h)
    for k in range(args.steps):
        b.step(STEPS_PER_SAMPLE)
        b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, args.warmup + args.steps + k)
    prof = B.gpe_profile_read(b.h)
    B.gpe_profile_enable(b.h, False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, ws)
    status = b.sync_status()
    value = su_per_step * args.steps * ws / (ms * 1e-3)

    # ensemble exchange: spectra summed over ranks, per-trajectory records gathered at their
    # global trajectory index (the layout of one batch of ws * 64 trajectories)
    acc_all = sharding.combine_accumulators(acc, nslots, nb, WL.ntraj, ws)
    assert acc_all.numel() == nslots * sharding.slot_doubles(nb, WL.ntraj * ws)

    # roofline of the dominant kernel class (bytes per launch: read + write of the 3-component field)
    peak, peak_kind = measured_peaks()
    dom = max(("xpass", "strided_pass"), key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    bytes_per_launch = 16.0 * WL.sites * 3 * WL.ntraj
    achieved = bytes_per_launch / (dom_ms / dom_n * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": ncu_traffic(dom), "kernel": dom, "peak_source": peak_kind,
                "avg_launch_us": dom_ms / dom_n * 1e3,
                "timing": "per-launch CUDA events over a second run of the same K bench steps",
                "classes_ms": {k: v[0] for k, v in prof.items() if v[1]},
                "classes_launches": {k: v[1] for k, v in prof.items() if v[1]},
                "effective_frac_16B_per_su": value / ws * 16.0 / (peak * 1e9)}

    # end to end through the API with host buffers: every bench step uploads its initial
    # fields from pinned host memory (gpe_batch_upload), runs the sampling interval and reads
    # its accumulator slot back (gpe_obs_download).  Two field buffers (two batches of the
    # same ensemble): the upload for step k + 1 runs on a copy stream while step k computes,
    # the way a pipelined caller would.
    host_psi = torch.empty_like(b.psi, device="cpu").pin_memory()
    host_psi.copy_(b.psi)
    host_acc = torch.empty(sd, dtype=torch.float64).pin_memory()
    b2 = B.GPEBatch(WL.shape, WL.ntraj, "c64", WL.c0, WL.c1, WL.q, WL.dt, dx=WL.dx)
    b2.set_traj_base(sharding.trajectory_base(rank, WL.ntraj))
    if args.no_autotune:
        b2.set_autotune(False)
    b2.psi.copy_(host_psi)
    b2.step(STEPS_PER_SAMPLE)   # first step: tile tuning
    bufs = (b, b2)
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in bufs]
    freed = [torch.cuda.Event() for _ in bufs]

    def put(k):
        i = k % 2
        cstream.wait_event(freed[i])   # the buffer's previous step has finished with it
        bufs[i].upload(host_psi, stream=cstream)
        copied[i].record(cstream)

    k_e2e = max(5, args.steps // 2)
    torch.cuda.synchronize()
    barrier(ws)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe = [torch.cuda.Event(enable_timing=True) for _ in range(k_e2e + 1)]
    f0.record(stream)
    fe[0].record(stream)
    cstream.wait_event(f0)
    put(0)
    for k in range(k_e2e):
        i = k % 2
        if k + 1 < k_e2e:
            put(k + 1)
        stream.wait_event(copied[i])
        bufs[i].step(STEPS_PER_SAMPLE)
        bufs[i].observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
        bufs[i].download_slot(acc, 0, host_acc, stream=stream)
        freed[i].record(stream)
        fe[k + 1].record(stream)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_steps = step_stats([fe[k].elapsed_time(fe[k + 1]) for k in range(k_e2e)])
    assert b2.sync_status() == B.GPE_OK
    b2.close()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), ws)
    e2e = {"value": su_per_step * k_e2e * ws / (e2e_ms * 1e-3), "unit": "site-updates/s",
           "h2d_bytes_per_step": int(b.psi.numel() * b.psi.element_size()),
           "d2h_bytes_per_step": int(sd * 8), "steps": k_e2e, "per_step": e2e_steps,
           "pipelined": "two field buffers; the next step's H2D copy overlaps the current step",
           "api": "C ABI with host buffers: gpe_batch_upload (pinned host fields -> batch), gpe_step_batch, "
                  "observables_accumulate, gpe_obs_download (accumulator slot -> pinned host)"}
    # An end-to-end rate above the device-only one can only be run-to-run noise (the e2e
    # region does strictly more work); flag it instead of reporting it silently.
    e2e["above_device_value"] = e2e["value"] > value
    if e2e["above_device_value"]:
        e2e["note"] = ("above the device-timed value by "
                       f"{100.0 * (e2e['value'] / value - 1.0):.2f} %: run-to-run noise of that size")
    tiles = b.tiles(0)
    lanes, xthreads = b.lanes(0), b.xpass_threads(0)
    b.close()

    # plain FP64 comparator: one trajectory per launch, no graph
    fp64 = None
    if rank == 0:
        pb = B.GPEBatch(WL.shape, 1, "c128", WL.c0, WL.c1, WL.q, WL.dt, dx=WL.dx)
        pb.init_noise(seed, WL.mean_spinor(), WL.noise_per_mode)
        pb.step(5)
        torch.cuda.synchronize()
        n64 = 40
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        pb.step(n64)
        g1.record(stream)
        torch.cuda.synchronize()
        v64 = WL.sites * 3 * n64 / (g0.elapsed_time(g1) * 1e-3)
        fp64 = {"value": v64, "unit": "site-updates/s", "ms_per_step": g0.elapsed_time(g1) / n64,
                "what": "complex128 fields, FP64 arithmetic, one 512^2 trajectory per launch, no graph",
                "fp32_batched_speedup": value / ws / v64}
        pb.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()

    # the ragged mix, measured after every leg of the headline number (one GPU only)
    secondary = None
    if rank == 0 and ws == 1 and not args.no_secondary:
        secondary = {"ragged": ragged_line(B, steps=3, warmup=2)}

    if rank == 0:
        out = {"metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": dict(workload_config(ws), column_tiles={"y": tiles[0], "autotuned": tiles[2]},
                              xpass_threads=xthreads, trajectory_lanes=lanes),
               "per_step": per_step, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
               "gpu_launches": launches, "fp64_plain": fp64, "status": status, "secondary": secondary}
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ncu_case():
    """Short run of the benchmark workload for ncu captures: noise, 4 steps, one observables call.
    The tile autotuner is off here so that the captured launches are the workload's own
    (the default width at 512 is the one the tuner keeps there; the bench line reports it),
    and the batch runs as one trajectory lane, so that each captured launch covers the whole
    batch like the per-kernel timings of the bench line."""
    from paper_2310_03636_gb300 import binding as B
    b = B.GPEBatch(WL.shape, WL.ntraj, "c64", WL.c0, WL.c1, WL.q, WL.dt, dx=WL.dx)
    b.set_autotune(False)
    b.set_lanes(1)
    b.init_noise(W.SEED_BASE, WL.mean_spinor(), WL.noise_per_mode)
    b.step(4)
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
    torch.cuda.synchronize()
    st = b.sync_status()
    b.close()
    print(json.dumps({"ncu_case": WL.name, "status": st}))
    if st != B.GPE_OK:
        sys.exit(1)


def run_other(args):
    """One JSON line for the other workload shapes (device-timed, no e2e/CPU legs)."""
    from paper_2310_03636_gb300 import binding as B
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    extra = {}
    if args.workload == "1d":
        wl = W.C1_1D
        b = B.GPEBatch(wl.shape, wl.ntraj, wl.dtype, wl.c0, wl.c1, wl.q, wl.dt, dx=wl.dx)
        per, flags = wl.sample_every, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG
        su = wl.site_updates_per_step * per
        name, dtype = wl.name, "f64"
    elif args.workload == "3d":
        wl = W.C3_3D[1]
        b = B.GPEBatch(wl.shape, wl.ntraj, wl.dtype, wl.c0, wl.c1, wl.q, wl.dt, dx=wl.dx)
        per, flags = wl.sample_every, B.GPE_OBS_DIAG
        su = wl.site_updates_per_step * per
        name, dtype = wl.name, "f32"
    elif args.workload == "ragged":
        shapes = W.ragged_sizes()
        b = B.GPEBatch(list(shapes), dtype="c64", c0=1.0, c1=-0.1, q=0.09, dt=0.02)
        b.set_graph(True)
        per, flags = 250, 0
        su = sum(int(np.prod(sh)) for sh in shapes) * 3 * per
        name, dtype = "ragged_200x1d_1k-16k_32x2d_128-1024_c64", "f32"
        extra["trajectories"] = len(shapes)
    elif args.workload in ("paper1d", "paper1d_f64"):
        # the paper's 1D grid (Sec. 2.2: 4096 points, three components), many runs at once
        f64 = args.workload == "paper1d_f64"
        ntraj = 304 if f64 else 3040
        b = B.GPEBatch((4096,), ntraj, "c128" if f64 else "c64", 1.0, -0.1, 0.09, 0.04)
        per, flags = (200 if f64 else 1000), 0
        su = 4096 * 3 * ntraj * per
        name, dtype = f"1d_4096_{'c128' if f64 else 'c64'}_{ntraj}traj", "f64" if f64 else "f32"
        extra["paper_context"] = ("paper: 4096 points, FP64, V100/A100, one 1.5e6-step run in 120-150 s "
                                  "with many runs per GPU (Sec. 2.2); not the same configuration")
    else:
        return run_adjoint(args)
    nb, sd = b.layout()
    acc = torch.zeros(max(1, args.warmup + args.steps) * max(sd, 1), dtype=torch.float64, device="cuda")
    b.init_noise(W.SEED_BASE, (0.0, 0.0, 1.0, 0.0, 0.0, 0.0), 0.5)
    for k in range(args.warmup):
        b.step(per)
        if flags:
            b.observables(acc, flags, k)
    torch.cuda.synchronize()
    l0 = B.gpe_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    e0.record(stream)
    for k in range(args.steps):
        b.step(per)
        if flags:
            b.observables(acc, flags, args.warmup + k)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if args.workload == "ragged":
        extra["scheduling"] = ragged_scheduling_bound(B, shapes, per, ms / args.steps)
    out = {"metric": "site-updates/s", "value": su * args.steps / (ms * 1e-3), "unit": "site-updates/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
           "config": {"workload": name, "steps_per_bench_step": per}, "clocks": clk,
           "gpu_launches": B.gpe_launch_count() - l0, "status": b.sync_status(), **extra}
    print(json.dumps(out), flush=True)
    b.close()


def ragged_line(B, steps, warmup):
    """The ragged mix (200 1D trajectories of 1024-16384 points and 32 2D ones of
    128^2-1024^2, FP32, graph replay), site-updates/s over 250-step intervals, and its
    perfect-packing bound."""
    stream = torch.cuda.current_stream()
    shapes = W.ragged_sizes()
    b = B.GPEBatch(list(shapes), dtype="c64", c0=1.0, c1=-0.1, q=0.09, dt=0.02)
    b.set_graph(True)
    per = 250
    su = sum(int(np.prod(sh)) for sh in shapes) * 3 * per
    b.init_noise(W.SEED_BASE, (0.0, 0.0, 1.0, 0.0, 0.0, 0.0), 0.5)
    for _ in range(warmup):
        b.step(per)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.step(per)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = b.sync_status()
    b.close()
    return {"workload": "ragged_200x1d_1k-16k_32x2d_128-1024_c64", "value": su / (ms * 1e-3),
            "unit": "site-updates/s", "ms_per_step": ms, "steps_per_bench_step": per, "trajectories": len(shapes),
            "status": st, "scheduling": ragged_scheduling_bound(B, shapes, per, ms)}


def fill_count(shape):
    """Trajectories of one shape that fill the GPU: at least 2.5e6 sites for 1D grids (every
    SM holds resident blocks) and 1.6e7 sites for 2D grids (passes of many full waves)."""
    sites = int(np.prod(shape))
    target = 2_500_000 if len(shape) == 1 else 16_000_000
    return max(1, -(-target // sites))


def ragged_scheduling_bound(B, shapes, per, measured_ms):
    """The mix against its shapes run one after another, each filling the GPU.  Each shape
    runs alone with enough trajectories to fill the GPU; the sum over shapes of the mix's
    work / that full-GPU rate is the time of a step interval scheduled shape by shape at each
    shape's best uniform rate -- what a single persistent kernel walking the shapes' work in
    turn would approach.  The concurrent streams can beat it (efficiency above 1) where
    shapes bound by different units (on-chip 1D kernels, 2D passes) overlap."""
    from collections import Counter
    per_shape = []
    ideal_s = 0.0
    for sh, cnt in sorted(Counter(shapes).items(), key=lambda kv: (len(kv[0]), kv[0])):
        nf = fill_count(sh)
        bb = B.GPEBatch(sh, nf, "c64", 1.0, -0.1, 0.09, 0.02)
        bb.init_noise(W.SEED_BASE, (0.0, 0.0, 1.0, 0.0, 0.0, 0.0), 0.5)
        bb.step(per)            # warm-up (and tile tuning)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record()
        for _ in range(reps):
            bb.step(per)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3 / reps
        bb.close()
        sites = int(np.prod(sh))
        rate = sites * 3 * per * nf / t
        work = sites * 3 * per * cnt
        ideal_s += work / rate
        per_shape.append({"shape": list(sh), "in_mix": cnt, "fill_trajectories": nf, "full_gpu_su_per_s": rate,
                          "ideal_ms": work / rate * 1e3})
    return {"measured_ms_per_step": measured_ms, "ideal_ms_per_step": ideal_s * 1e3,
            "packing_efficiency": ideal_s * 1e3 / measured_ms, "per_shape": per_shape,
            "note": "ideal = sum over shapes of (the mix's work of that shape / its full-GPU rate), "
                    "i.e. the shapes run one after another each filling the GPU"}


def run_adjoint(args):
    """Gradient of the late-time S_perp band loss w.r.t. 64 q knots and the initial fields:
    2D 256^2 x 8 trajectories, 4096 steps, checkpoints every 256 (forward + recompute +
    reverse sweep).  site-updates counted for the forward steps only."""
    from paper_2310_03636_gb300 import binding as B
    from paper_2310_03636_gb300.adjoint import AdjointConfig, sf_loss
    torch.cuda.set_device(0)
    wl = W.C5_ADJ
    cfg = AdjointConfig(wl.shape, wl.steps, wl.dt, t_end=wl.steps * wl.dt, kmin=0.2, kmax=0.4, c0=wl.c0, c1=wl.c1,
                        dtype="c64", checkpoint_every=256)
    b = B.GPEBatch(wl.shape, wl.ntraj, "c64", wl.c0, wl.c1, wl.q, wl.dt)
    b.init_noise(W.SEED_BASE + 5, wl.mean_spinor(), wl.noise_per_mode)
    psi0 = b.psi.clone()
    b.close()
    knots = torch.tensor(W.q_ramp_knots(64), dtype=torch.float64)

    def once():
        k = knots.clone().requires_grad_(True)
        p = psi0.clone().requires_grad_(True)
        sf_loss(k, p, cfg).backward()
    for _ in range(max(1, args.warmup // 3)):
        once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = max(1, args.steps // 10)
    for _ in range(n):
        once()
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / n
    su = wl.site_updates_per_step * wl.steps
    print(json.dumps({"metric": "site-updates/s (forward steps of one gradient)", "value": su / el,
                      "unit": "site-updates/s", "n_gpus": 1, "steps": n, "warmup": max(1, args.warmup // 3),
                      "ms_per_step": el * 1e3, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": wl.name, "knots": 64, "checkpoint_every": 256}}), flush=True)


def alu_peaks():
    """FMA throughput (best of 3 launches per kind) with the SM clocks seen meanwhile."""
    import torch
    from paper_2310_03636_gb300 import binding as B
    torch.cuda.init()
    kinds = {"fp32_fma": (0, 1 << 16), "fp32x2_fma": (1, 1 << 15), "fp64_fma": (2, 1 << 10)}
    out = {}
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    for name, (kind, iters) in kinds.items():
        out[name + "_tflops"] = max(B.gpe_fma_rate(kind, iters) for _ in range(3)) / 1e12
    out["clocks"] = clk.stop()
    print(json.dumps({"alu_peaks": out, "sms": torch.cuda.get_device_properties(0).multi_processor_count}),
          flush=True)


def main():
    args = parse()
    if args.alu_peaks:
        alu_peaks()
    elif args.ncu_case:
        ncu_case()
    elif args.workload != "2d":
        run_other(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
