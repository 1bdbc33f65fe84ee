"""Philox4x32-10 counter-based generator and the truncated-Wigner noise draw (oracle side).

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by ``__graft_entry__.smoke()`` and
by the CPU-baseline / reference leg of ``bench.py``; the CUDA library never uses it.

The generator is written from its published definition: J. K. Salmon, M. A. Moraes,
R. O. Dror and D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11
(Philox-4x32 with R = 10 rounds).  One round maps the counter (c0, c1, c2, c3) with
key (k0, k1) to

    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0)),

with M0 = 0xD2511F53, M1 = 0xCD9E8D57, and the key is bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85) between rounds.

The paper (Sec. 2.2) only says that runs start from "slightly fluctuating" initial
conditions to represent quantum fluctuations; the noise model here (complex Gaussian,
1/2 particle per mode, drawn site by site through Box-Muller) is this build's reading.
The GPU library implements the same integer stream independently, so both sides draw
identical noise from the same seed.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """Philox4x32-10 of Salmon et al. (SC'11).

    counter: tuple of four uint32-valued arrays (broadcastable), key: tuple of two.
    Returns four uint64 arrays holding the 32-bit output words.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in counter)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & MASK32 for k in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniforms_from_words(w0, w1, w2, w3):
    """Two FP64 uniforms from the four 32-bit words.

    u1 in (0, 1] from the 64-bit integer (w1 << 32 | w0), u2 in [0, 1) from
    (w3 << 32 | w2); both keep the top 53 bits.
    """
    x1 = (np.asarray(w1, np.uint64) << np.uint64(32)) | np.asarray(w0, np.uint64)
    x2 = (np.asarray(w3, np.uint64) << np.uint64(32)) | np.asarray(w2, np.uint64)
    scale = 2.0 ** -53
    u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * scale
    u2 = (x2 >> np.uint64(11)).astype(np.float64) * scale
    return u1, u2


def tw_noise(shape, seed, traj, noise_per_mode, dx):
    """Complex Gaussian truncated-Wigner noise eta_m(x) for one trajectory.

    shape: spatial shape (z, y, x order, fastest last).  Returns complex128 of shape
    (3, *shape).  Counter for component m (0, 1, 2 <-> psi_1, psi_0, psi_-1) at flat
    site index s of trajectory ``traj``: (s mod 2^32, m, traj, s >> 32); key = (seed
    low word, seed high word).  Box-Muller: eta = sqrt(-ln u1) e^{2 pi i u2} sigma with
    sigma^2 = noise_per_mode / dx^d, so <|eta|^2> = noise_per_mode / dx^d.  A unitary
    DFT maps iid complex Gaussians onto iid ones, so every plane-wave mode then carries
    ``noise_per_mode`` particles on average.
    """
    d = len(shape)
    nsite = int(np.prod(shape))
    s = np.arange(nsite, dtype=np.uint64)
    seed = int(seed)
    key = (np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    sigma = np.sqrt(noise_per_mode / dx ** d)
    out = np.empty((3, nsite), dtype=np.complex128)
    for m in range(3):
        w = philox4x32_10((s & MASK32, np.uint64(m), np.uint64(traj), s >> np.uint64(32)), key)
        u1, u2 = uniforms_from_words(*w)
        r = np.sqrt(-np.log(u1)) * sigma
        out[m] = r * np.exp(2j * np.pi * u2)
    return out.reshape((3,) + tuple(shape))
