"""Seeded synthetic workloads and test fields (inputs only; none of the method's arithmetic).

Both the CUDA path (through the binding) and the CPU oracle receive the arrays made here.
Random test fields use numpy's Philox bit generator; the truncated-Wigner noise itself is
drawn inside ``tw_init_noise`` from a seed, not here.

The workload shapes follow the paper's own simulation sizes (Sec. 2.2: 1D grids of
4096 points, 3D grids up to 256^3 x 3 complex components, many runs per GPU) and the
parameter set of a ferromagnetic spin-1 quench from the polar state.
"""
from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 20231005


@dataclass(frozen=True)
class Workload:
    name: str
    shape: tuple            # spatial shape, slowest axis first ((nx,), (ny, nx), (nz, ny, nx))
    ntraj: int
    dtype: str              # "c64" or "c128"
    c0: float = 1.0
    c1: float = -0.1
    q: float = 0.09         # 0.9 n |c1| with n = 1
    n: float = 1.0          # condensate density (polar state: all atoms in m = 0)
    dt: float = 0.02
    steps: int = 1000
    sample_every: int = 0   # 0: no sampling
    dx: float = 1.0
    noise_per_mode: float = 0.5

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def sites(self):
        return math.prod(self.shape)

    @property
    def site_updates_per_step(self):
        """points x 3 components x trajectories (one time step)."""
        return self.sites * 3 * self.ntraj

    def mean_spinor(self):
        """(re, im) of (psi_1, psi_0, psi_-1): polar state sqrt(n) in m = 0."""
        return (0.0, 0.0, math.sqrt(self.n), 0.0, 0.0, 0.0)


C1_1D = Workload("1d_n256_c128_1traj", (256,), 1, "c128", dt=0.01, steps=1000, sample_every=100)
C2_2D = Workload("2d_512x512_c64_64traj", (512, 512), 64, "c64", dt=0.02, steps=10000,
                 sample_every=250)
C3_3D = tuple(
    Workload(f"3d_256cube_c64_8traj_q{f:.1f}", (256, 256, 256), 8, "c64", q=f * 0.1,
             dt=0.02, steps=2000, sample_every=100)
    for f in (0.3, 0.9, 1.5))
C5_ADJ = Workload("adjoint_2d_256x256_c64_8traj", (256, 256), 8, "c64", dt=0.02, steps=4096)
PAPER_1D = Workload("1d_n4096_c64", (4096,), 1, "c64", dt=0.01, steps=1500000)


def ragged_sizes(seed=42, n1d=200, n2d=32):
    """Mixed batch: n1d 1D trajectories with N uniform over {2^10 .. 2^14} and n2d 2D
    trajectories with side uniform over {128, 256, 512, 1024}, drawn with Philox(seed)."""
    g = np.random.Generator(np.random.Philox(seed))
    n1 = [int(2 ** e) for e in g.integers(10, 15, size=n1d)]
    n2 = [int(s) for s in g.choice([128, 256, 512, 1024], size=n2d)]
    return [(n,) for n in n1] + [(s, s) for s in n2]


def q_ramp_knots(nknots=64, q_start=0.2, q_end=0.05):
    """q(t) knots of a linear ramp (values already in units of n|c1| x n|c1| = 0.1)."""
    return np.linspace(q_start, q_end, nknots)


def random_field(shape, ntraj, seed, scale=1.0, mean=(0.0, 1.0, 0.0)):
    """Seeded complex test field of shape (ntraj, 3, *shape): mean spinor + scale * N(0,1)."""
    g = np.random.Generator(np.random.Philox(seed))
    z = g.standard_normal((ntraj, 3) + tuple(shape)) + 1j * g.standard_normal((ntraj, 3) + tuple(shape))
    m = np.asarray(mean, dtype=np.complex128).reshape((1, 3) + (1,) * len(shape))
    return m + scale * z / math.sqrt(2.0)


def smooth_random_field(shape, ntraj, seed, kmax_frac=0.25, amp=0.3, mean=(0.2, 1.0, 0.1)):
    """Seeded band-limited test field: random Fourier modes with |j| <= kmax_frac * n/2."""
    g = np.random.Generator(np.random.Philox(seed))
    d = len(shape)
    spec = g.standard_normal((ntraj, 3) + tuple(shape)) + 1j * g.standard_normal((ntraj, 3) + tuple(shape))
    mask = np.ones(shape, dtype=bool)
    for ax, n in enumerate(shape):
        j = np.fft.fftfreq(n, d=1.0 / n)
        view = [1] * d
        view[ax] = n
        mask = mask & (np.abs(j).reshape(view) <= kmax_frac * n / 2)
    spec = spec * mask
    f = np.fft.ifftn(spec, axes=tuple(range(2, 2 + d)))
    f = f / max(np.abs(f).max(), 1e-300) * amp
    m = np.asarray(mean, dtype=np.complex128).reshape((1, 3) + (1,) * d)
    return m + f


def smooth_potential(shape, seed, amp=0.5, dx=1.0, spread=0.2):
    """Seeded real test potential V_m(x), shape (3, *shape): a periodic cosine well
    amp * sum_a (1 - cos(2 pi x_a / L_a)) common to the three components, plus a
    band-limited random part of relative size ``spread`` that differs per component."""
    d = len(shape)
    base = np.zeros(shape)
    for ax, n in enumerate(shape):
        x = np.arange(n) * dx
        view = [1] * d
        view[ax] = n
        base = base + (1.0 - np.cos(2 * np.pi * x / (n * dx))).reshape(view)
    rnd = smooth_random_field(shape, 1, seed, kmax_frac=0.125, amp=1.0, mean=(0.0, 0.0, 0.0))[0].real
    return amp * (base[None] + spread * rnd)


def plane_wave(shape, js, dx=1.0):
    """exp(i k.x) with k_a = 2 pi j_a / (n_a dx); js ordered like shape."""
    d = len(shape)
    ph = np.zeros(shape)
    for ax, (n, j) in enumerate(zip(shape, js)):
        x = np.arange(n) * dx
        view = [1] * d
        view[ax] = n
        ph = ph + (2 * np.pi * j / (n * dx) * x).reshape(view)
    return np.exp(1j * ph)
