"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the same seeded
inputs.  Tolerances: per-component relative L2 error <= 1e-11 (FP64 fields) and <= 1e-4
(FP32 fields) after 200 steps; ensemble spectra within 1e-3 relative (FP32), 1e-10 (FP64).
"""
import math

import numpy as np
import pytest
import torch

from oracle import gpe_oracle as O
from oracle.philox import tw_noise
from paper_2310_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C0, C1, Q = 1.0, -0.1, 0.09
MEAN = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_03636_gb300 import binding
    return binding


def oracle_initial(shape, ntraj, seed, dx=1.0, npm=0.5, mean=MEAN, ids=None):
    ids = range(ntraj) if ids is None else ids
    out = []
    for t in ids:
        eta = tw_noise(shape, seed, t, npm, dx)
        for m in range(3):
            eta[m] += mean[2 * m] + 1j * mean[2 * m + 1]
        out.append(eta)
    return np.stack(out)


def rel_l2_per_comp(gpu, ref):
    """max over trajectories and components of ||gpu - ref|| / ||ref||."""
    d = len(gpu.shape) - 2
    ax = tuple(range(2, 2 + d))
    num = np.sqrt((np.abs(gpu - ref) ** 2).sum(axis=ax))
    den = np.sqrt((np.abs(ref) ** 2).sum(axis=ax))
    return float((num / den).max())


def run_oracle(psi0, dt, steps, d, c0=C0, c1=C1, q=Q, dx=1.0, t0=0.0):
    return O.propagate(torch.as_tensor(psi0), dt, steps, c0, c1, q, dx, d, t0=t0).numpy()


# ------------------------------------------------------------------ noise

@pytest.mark.parametrize("dtype,shape,dx", [("c128", (64, 128), 1.0), ("c64", (256,), 0.5), ("c128", (64, 64, 64), 0.7)])
def test_noise_matches_oracle(B, dtype, shape, dx):
    b = B.GPEBatch(shape, 3, dtype, dx=dx)
    mean = (0.1, -0.2, 0.9, 0.05, 0.0, 0.3)
    b.init_noise(987654321012345, mean, 0.5)
    gpu = b.psi.cpu().numpy()
    ref = oracle_initial(shape, 3, 987654321012345, dx=dx, mean=mean)
    tol = 1e-13 if dtype == "c128" else 2e-7
    assert np.abs(gpu - ref).max() < tol * max(1.0, np.abs(ref).max())
    b.close()


# ------------------------------------------------------------------ propagation, FP64

@pytest.mark.parametrize("shape,ntraj,dt,steps", [
    ((256,), 1, 0.01, 200),          # 1D N = 256, one trajectory, dt = 0.01
    ((64,), 3, 0.02, 150),
    ((2048,), 2, 0.02, 60),
    ((64, 128), 2, 0.02, 200),       # non-square 2D: transposed axes would fail
    ((128, 64), 1, 0.02, 40),
    ((64, 64, 128), 1, 0.02, 12),    # 3D with three distinct pass kinds
])
def test_propagation_fp64(B, shape, ntraj, dt, steps):
    seed = 4242
    b = B.GPEBatch(shape, ntraj, "c128", C0, C1, Q, dt)
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy()
    ref = run_oracle(oracle_initial(shape, ntraj, seed), dt, steps, len(shape))
    err = rel_l2_per_comp(gpu, ref)
    assert err <= 1e-11, err
    b.close()


@pytest.mark.parametrize("shape,ntraj,steps", [((256,), 2, 200), ((2048,), 2, 200), ((4096,), 2, 200), ((128, 128), 4, 200),
                                         ((64, 64, 64), 1, 50)])
def test_propagation_fp32(B, shape, ntraj, steps):
    seed, dt = 77, 0.02
    b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, dt)
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial(shape, ntraj, seed), dt, steps, len(shape))
    err = rel_l2_per_comp(gpu, ref)
    assert err <= 1e-4, err
    b.close()


def test_propagation_fp32_3d_200_steps(B):
    """FP32 3D at the 200-step bar: the x pass and the tensor-map y and z passes (the z pass
    is its own kernel) against the oracle, per component."""
    shape, ntraj, steps, dt, seed = (64, 64, 64), 2, 200, 0.02, 78
    b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, dt)
    assert b.tiles(0)[1] != 0      # the contiguous batch takes the tensor-map z pass
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial(shape, ntraj, seed), dt, steps, 3)
    err = rel_l2_per_comp(gpu, ref)
    assert err <= 1e-4, err
    b.close()


@pytest.mark.parametrize("dtype,shape,steps,tol", [
    ("c64", (1024, 1024), 20, 1e-4),      # largest x and y extents
    ("c128", (1024, 1024), 8, 1e-11),
    ("c64", (64, 64, 1024), 6, 1e-4),     # largest z extent (tensor-map z pass)
    ("c64", (1024, 64, 64), 6, 1e-4),     # largest x extent in 3D
])
def test_maximum_grids_vs_oracle(B, dtype, shape, steps, tol):
    """The largest extent each pass accepts (1024 points per axis), one trajectory, element
    by element against the oracle."""
    seed, dt = 31, 0.02
    b = B.GPEBatch(shape, 1, dtype, C0, C1, Q, dt)
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial(shape, 1, seed), dt, steps, len(shape))
    assert rel_l2_per_comp(gpu, ref) <= tol
    b.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("shape", [(256,), (64, 128), (64, 64, 64)])
def test_single_component_states_keep_closed_form(B, dtype, shape):
    """Degenerate states of Eq. (GPE) with a closed form: a uniform field in one component
    only.  Then a = psi_-1^* psi_0 = 0 and b = psi_0^* psi_1 = 0, so the spin-mixing step is
    the identity and the empty components stay exactly zero, and the occupied one turns at
    its mean-field rate: f_0 = (c0 + c1) rho - c1 |psi_0|^2 = c0 rho for m = 0, and
    f_1 = q + (c0 + c1) rho - 2 c1 |psi_-1|^2 = q + (c0 + c1) rho for m = +1 (kinetic factor 1:
    only the k = 0 mode is occupied).  The rotation integrator must agree."""
    dt, steps, rho = 0.02, 200, 1.3
    tol = 2e-5 if dtype == "c64" else 1e-12
    n = int(np.prod(shape))
    for occ, rate in ((1, C0 * rho), (0, Q + (C0 + C1) * rho)):
        for integrator in (0, 1):
            b = B.GPEBatch(shape, 2, dtype, C0, C1, Q, dt)
            b.set_integrator(integrator)
            psi = torch.zeros_like(b.psi)
            psi[:, occ] = math.sqrt(rho)
            b.psi.copy_(psi)
            b.step(steps)
            assert b.sync_status() == B.GPE_OK
            out = b.psi.cpu().numpy().astype(np.complex128)
            empty = [m for m in range(3) if m != occ]
            assert np.all(out[:, empty] == 0), "empty components must stay exactly zero"
            want = math.sqrt(rho) * np.exp(-1j * rate * dt * steps)
            err = np.abs(out[:, occ].reshape(2, n) - want).max() / math.sqrt(rho)
            assert err <= tol, (occ, integrator, err)
            b.close()


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-4), ("c128", 1e-11)])
def test_no_spin_coupling(B, dtype, tol):
    """c1 = 0: the spin-mixing step has a zero coupling (its series coefficients at u = 0) and
    the D step loses its spin terms; noisy fields against the oracle with the same c1."""
    shape, ntraj, steps, dt, seed = (64, 128), 2, 100, 0.02, 5
    b = B.GPEBatch(shape, ntraj, dtype, C0, 0.0, Q, dt)
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial(shape, ntraj, seed), dt, steps, 2, c1=0.0)
    assert rel_l2_per_comp(gpu, ref) <= tol
    b.close()


@pytest.mark.parametrize("shape", [(64, 128), (32 * 4, 512)])
def test_fp32_kinetic_angles_beyond_half_pi(B, shape):
    """dt and dx with kinetic phases dt k^2/2 up to 2 rad at the largest k: the tables then
    carry a sign per entry and the x pass reads them from global memory (no compact
    table); same parity bar, and the x-pass block size is not selectable there.  Weak
    couplings and noise keep the nonlinear phases small (with c0 = 1 and 2 particles per
    site at dx = 1/2 they reach ~1 rad per step and the chaotic growth of rounding errors,
    the same in FP64, dominates after a few tens of such steps)."""
    dx, dt, steps, seed = 0.5, 0.1, 40, 12
    c0, c1 = 0.1, -0.01
    b = B.GPEBatch(shape, 2, "c64", c0, c1, Q, dt, dx=dx)
    b.init_noise(seed, MEAN, 0.05)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial(shape, 2, seed, dx=dx, npm=0.05), dt, steps, 2, c0=c0, c1=c1, dx=dx)
    assert rel_l2_per_comp(gpu, ref) <= 1e-4
    with pytest.raises(B.GPEError) as ei:
        b.set_xpass_threads(128)
    assert ei.value.status == B.GPE_EUNSUPPORTED
    b.close()


def test_split_calls_and_time_dependent_q(B):
    """q(t) ramp through knots, advanced in uneven chunks: same as the oracle's single run."""
    shape, ntraj, dt, seed = (64, 64), 2, 0.02, 5
    knots = np.linspace(0.2, 0.05, 7)
    t_end = 60 * dt
    b = B.GPEBatch(shape, ntraj, "c128", C0, C1, Q, dt, q_knots=knots, t_end=t_end)
    b.init_noise(seed, MEAN, 0.5)
    for n in (1, 17, 0, 30, 12):
        b.step(n)
    assert b.step_count == 60
    gpu = b.psi.cpu().numpy()
    qf = O.q_piecewise_linear(torch.as_tensor(knots), t_end)
    ref = O.propagate(torch.as_tensor(oracle_initial(shape, ntraj, seed)), dt, 60, C0, C1, qf, 1.0, 2).numpy()
    assert rel_l2_per_comp(gpu, ref) <= 1e-11
    b.close()


def test_1d_time_dependent_q(B):
    shape, dt, seed = (512,), 0.01, 8
    knots = [0.3, 0.0, 0.2]
    b = B.GPEBatch(shape, 2, "c128", C0, C1, Q, dt, q_knots=knots, t_end=1.0)
    b.init_noise(seed, MEAN, 0.5)
    b.step(70)
    b.step(50)
    gpu = b.psi.cpu().numpy()
    qf = O.q_piecewise_linear(torch.as_tensor(knots, dtype=torch.float64), 1.0)
    ref = O.propagate(torch.as_tensor(oracle_initial(shape, 2, seed)), dt, 120, C0, C1, qf, 1.0, 1).numpy()
    assert rel_l2_per_comp(gpu, ref) <= 1e-11
    b.close()


def test_smooth_field_dx_and_couplings(B):
    """A caller-written initial field, dx != 1, other couplings (c1 > 0)."""
    shape, dx, dt = (64, 128), 0.6, 0.015
    psi0 = W.smooth_random_field(shape, 2, seed=19)
    c0, c1, q = 0.7, 0.35, -0.05
    psi = torch.as_tensor(psi0).to("cuda")
    b = B.GPEBatch(shape, 2, "c128", c0, c1, q, dt, dx=dx, psi=psi.contiguous())
    b.step(80)
    ref = run_oracle(psi0, dt, 80, 2, c0, c1, q, dx)
    assert rel_l2_per_comp(b.psi.cpu().numpy(), ref) <= 1e-11
    b.close()


def test_ragged_batch(B):
    """Trajectories of different shapes in one batch, each matches the oracle; spectra per
    shape group (one block per group in the slot) and per-trajectory diagnostics match the
    oracle's, a group with unequal sides adds diagnostics but no spectra."""
    shapes = [(256,), (64, 64), (128,), (64, 64), (64, 128), (8192,)]
    b = B.GPEBatch(list(shapes), dtype="c128", dt=0.02)
    b.init_noise(31, MEAN, 0.5)
    b.step(40)
    for i, s in enumerate(shapes):
        ref = run_oracle(oracle_initial(s, 1, 31, ids=[i]), 0.02, 40, len(s))
        assert rel_l2_per_comp(b.psi[i].cpu().numpy()[None], ref) <= 1e-11
    nb, sd = b.layout()
    nt = len(shapes)
    assert sd == 4 * nb + 9 * nt
    # bins: 1D 256 -> 129, 2D 64^2 -> 46, 1D 128 -> 65, 64 x 128 none, 1D 8192 -> 4097
    assert nb == 129 + 46 + 65 + 4097
    acc = torch.zeros(sd, dtype=torch.float64, device="cuda")
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
    assert b.sync_status() == B.GPE_OK
    a = acc.cpu().numpy()
    counts = b.bin_counts()
    groups = {}
    for i, s in enumerate(shapes):
        groups.setdefault(s, []).append(i)
    for s, ids in groups.items():
        gnb, off = b.group_layout(ids[0])
        if len(set(s)) > 1:
            assert gnb == 0
            continue
        psi = np.stack([b.psi[i].cpu().numpy() for i in ids])
        rs, _, rc = oracle_observables(psi, 1.0, len(s))
        assert gnb == rs.shape[1]
        got = a[off:off + 4 * gnb].reshape(4, gnb)
        np.testing.assert_array_equal(counts[off // 4:off // 4 + gnb], rc)
        assert np.abs(got - rs).max() <= 1e-10 * np.abs(rs).max(), s
    diag = a[4 * nb:4 * nb + 8 * nt].reshape(nt, 8)
    for i, s in enumerate(shapes):
        p = torch.as_tensor(b.psi[i].cpu().numpy())
        ref = O.diagnostics(p, 1.0, C0, C1, Q, len(s)).numpy()
        np.testing.assert_allclose(diag[i], ref, rtol=1e-10, atol=1e-9)
    b.close()
    # no group with equal sides: spectra refused
    b = B.GPEBatch([(64, 128), (128, 64)], dtype="c128", dt=0.02)
    acc = b.new_accumulator(1)
    with pytest.raises(B.GPEError) as ei:
        b.observables(acc, B.GPE_OBS_SPECTRA, 0)
    assert ei.value.status == B.GPE_EUNSUPPORTED
    b.close()


# ------------------------------------------------------------------ observables

def oracle_observables(psi, dx, d, q=Q):
    """Spectra summed over trajectories per radial bin, and per-trajectory diagnostics."""
    p = torch.as_tensor(psi)
    shape = psi.shape[2:]
    bins = O.radial_bins(shape)
    nk = O.bin_sum(O.occupation_modes(p, dx, d), bins).sum(0).numpy()      # (3, nb)
    sk = O.bin_sum(O.spin_structure_modes(p, dx, d), bins).sum(0).numpy()  # (nb,)
    spec = np.concatenate([nk, sk[None]], 0)
    diag = O.diagnostics(p, dx, C0, C1, q, d).numpy()
    return spec, diag, O.bin_counts(shape).numpy()


@pytest.mark.parametrize("dtype,shape,ntraj,dx,steps", [
    ("c128", (256,), 1, 1.0, 100),
    ("c128", (128, 128), 3, 0.8, 30),
    ("c64", (128, 128), 4, 1.0, 30),
    ("c128", (64, 64, 64), 2, 1.0, 5),
    # 1D grids on thread-block clusters: spectra through the four-step transform
    ("c128", (4096,), 2, 1.0, 20),          # FP64 cluster of 2 x 2048
    ("c128", (16384,), 1, 0.7, 10),         # FP64 cluster of 8 x 2048
    ("c64", (8192,), 2, 1.0, 20),           # FP32 cluster of 2 x 4096
    ("c64", (32768,), 2, 1.0, 10),          # FP32 cluster of 8 x 4096
])
def test_observables(B, dtype, shape, ntraj, dx, steps):
    b = B.GPEBatch(shape, ntraj, dtype, C0, C1, Q, 0.02, dx=dx)
    b.init_noise(11, MEAN, 0.5)
    b.step(steps)
    nb, sd = b.layout()
    acc = b.new_accumulator(3)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 1)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 1)     # accumulates: x2
    assert b.sync_status() == B.GPE_OK
    a = acc.cpu().numpy()
    assert np.all(a[:sd] == 0) and np.all(a[2 * sd:] == 0)
    spec, diag = B.unpack_slot(a[sd:2 * sd], nb, ntraj)
    psi = b.psi.cpu().numpy().astype(np.complex128)
    rs, rd, counts = oracle_observables(psi, dx, len(shape))
    np.testing.assert_array_equal(b.bin_counts(), counts)
    tol = 1e-10 if dtype == "c128" else 1e-5
    scale = np.abs(rs).max(axis=1, keepdims=True)
    assert np.abs(spec / 2 - rs).max() <= tol * scale.max()
    np.testing.assert_allclose(diag / 2, rd, rtol=tol, atol=tol * np.abs(rd).max())
    # deterministic: a second identical accumulation gives bitwise identical sums
    acc2 = b.new_accumulator(3)
    b.observables(acc2, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 1)
    b.observables(acc2, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 1)
    assert torch.equal(acc, acc2)
    b.close()


def test_spectra_fp32_vs_oracle_ensemble(B):
    """FP32 fields, ensemble spectra within 1e-3 relative of the FP64 oracle run."""
    shape, ntraj, steps, dt, seed = (128, 128), 8, 200, 0.02, 3
    b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, dt)
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    nb, sd = b.layout()
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_SPECTRA, 0)
    spec, _ = B.unpack_slot(acc, nb, ntraj)
    ref_psi = run_oracle(oracle_initial(shape, ntraj, seed), dt, steps, 2)
    rs, _, counts = oracle_observables(ref_psi, 1.0, 2)
    # compare the bin means of S_perp and of |A_m|^2 (n_m + 1/2)
    cnt = counts * ntraj
    gS, rS = spec[3] / cnt, rs[3] / cnt
    assert np.abs(gS - rS).max() / np.abs(rS).max() <= 1e-3
    gN, rN = spec[:3] / cnt + 0.5, rs[:3] / cnt + 0.5
    assert (np.abs(gN - rN) / np.abs(rN)).max() <= 1e-3
    b.close()


def test_spectra_fp32_512_vs_oracle(B):
    """FP32 fields on the benchmark grid (512^2): the spectra kernels the bench runs at this
    size (row FFT, column FFT, radial bins) against the oracle's binned spectra after 200
    steps, bin means within 1e-3 relative, and the FP64 diagnostics."""
    wl = W.C2_2D
    ntraj, steps, seed = 4, 200, W.SEED_BASE
    b = B.GPEBatch(wl.shape, ntraj, "c64", wl.c0, wl.c1, wl.q, wl.dt)
    b.init_noise(seed, wl.mean_spinor(), wl.noise_per_mode)
    b.step(steps)
    nb, sd = b.layout()
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
    assert b.sync_status() == B.GPE_OK
    spec, diag = B.unpack_slot(acc, nb, ntraj)
    ref_psi = run_oracle(oracle_initial(wl.shape, ntraj, seed), wl.dt, steps, 2, wl.c0, wl.c1, wl.q)
    rs, rd, counts = oracle_observables(ref_psi, 1.0, 2, q=wl.q)
    assert nb == 363
    np.testing.assert_array_equal(b.bin_counts(), counts)
    cnt = counts * ntraj
    gS, rS = spec[3] / cnt, rs[3] / cnt
    assert np.abs(gS - rS).max() / np.abs(rS).max() <= 1e-3
    gN, rN = spec[:3] / cnt + 0.5, rs[:3] / cnt + 0.5
    assert (np.abs(gN - rN) / np.abs(rN)).max() <= 1e-3
    np.testing.assert_allclose(diag[:, :3], rd[:, :3], rtol=1e-4)
    b.close()


# ------------------------------------------------------------------ edge cases and errors

def test_zero_steps_is_noop(B):
    b = B.GPEBatch((64, 64), 1, "c64")
    b.init_noise(1, MEAN, 0.5)
    before = b.psi.clone()
    b.step(0)
    torch.cuda.synchronize()
    assert torch.equal(before, b.psi)
    b.close()


def test_invalid_arguments(B):
    psi = torch.zeros((3, 64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(B.GPEError) as e:      # an empty batch
        B.gpe_batch_create([], B.GPE_C64, 1, -0.1, 0.09, 0.02)
    assert e.value.status == B.GPE_EINVAL
    with pytest.raises(B.GPEError) as e:
        B.gpe_batch_create([((64, 60), 1.0, psi)], B.GPE_C64, 1, -0.1, 0.09, 0.02)
    assert e.value.status == B.GPE_EINVAL
    with pytest.raises(B.GPEError) as e:
        B.gpe_batch_create([((64, 64), 1.0, psi)], B.GPE_C64, 1, -0.1, 0.09, -0.02)
    assert e.value.status == B.GPE_EINVAL
    big = torch.zeros((3, 2048, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(B.GPEError) as e:
        B.gpe_batch_create([((2048, 64), 1.0, big)], B.GPE_C64, 1, -0.1, 0.09, 0.02)
    assert e.value.status == B.GPE_EUNSUPPORTED
    b = B.GPEBatch((64, 64), 1, "c64")
    with pytest.raises(B.GPEError) as e:
        b.step(-1)
    assert e.value.status == B.GPE_EINVAL
    acc = b.new_accumulator(1)
    with pytest.raises(B.GPEError) as e:
        b.observables(acc, 0x10, 0)
    assert e.value.status == B.GPE_EINVAL
    b.close()


def test_nonfinite_is_reported(B):
    """A NaN in the field is caught by the FP64 diagnostics reduction (status word)."""
    b = B.GPEBatch((64, 64), 1, "c64")
    b.init_noise(2, MEAN, 0.5)
    b.psi[0, 1, 3, 5] = float("nan")
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_DIAG, 0)
    assert b.sync_status() == B.GPE_ENONFINITE
    assert b.sync_status() == B.GPE_OK      # cleared
    b.close()


# ------------------------------------------------------------------ full size, sampled

def test_full_size_2d_512_sampled(B):
    """The 2D 512^2 x 64-trajectory FP32 workload in the launch configuration the bench
    times; sampled trajectories checked against the oracle after 200 steps."""
    wl = W.C2_2D
    b = B.GPEBatch(wl.shape, wl.ntraj, "c64", wl.c0, wl.c1, wl.q, wl.dt)
    seed = W.SEED_BASE
    b.init_noise(seed, wl.mean_spinor(), wl.noise_per_mode)
    b.step(200)
    assert b.sync_status() == B.GPE_OK
    for t in (0, 63):
        gpu = b.psi[t:t + 1].cpu().numpy().astype(np.complex128)
        ref = run_oracle(oracle_initial(wl.shape, 1, seed, ids=[t]), wl.dt, 200, 2)
        assert rel_l2_per_comp(gpu, ref) <= 1e-4
    b.close()


def test_own_sincos_against_cuda(B):
    """The local step's FP32 sin/cos (Cody-Waite + Taylor) stays within 2 ulp-scale of
    CUDA's sincosf and of the FP64 value, over small, typical and large arguments."""
    g = torch.Generator().manual_seed(3)
    xs = torch.cat([torch.linspace(-4, 4, 200001), (torch.rand(200000, generator=g) - 0.5) * 2e4,
                    torch.tensor([0.0, -0.0, 1e-30, 1e4, -1e4, 3e4, 1e6, float(np.pi) / 4, 1e-6])]).float()
    out = B.gpe_check_sincos(xs.cuda()).cpu().double()
    x64 = xs.double()
    s_ref, c_ref = torch.sin(x64), torch.cos(x64)
    assert (out[:, 0] - s_ref).abs().max() < 3e-7 * max(1.0, 1.0)
    assert (out[:, 1] - c_ref).abs().max() < 3e-7
    # relative accuracy of sin for small arguments (the common case in the local step)
    small = xs.abs() < 0.5
    rel = ((out[small, 0] - s_ref[small]).abs() / s_ref[small].abs().clamp_min(1e-30))
    assert rel.max() < 2.5e-7
    # never worse than the library by more than 1.5e-7 absolute
    assert (out[:, 0] - s_ref).abs().max() <= (out[:, 2] - s_ref).abs().max() + 1.5e-7
    assert (out[:, 1] - c_ref).abs().max() <= (out[:, 3] - c_ref).abs().max() + 1.5e-7


def test_fma_rate_probe(B):
    """The arithmetic-rate probe returns finite, ordered rates: FP32 above FP64, and below
    what 152 SMs x 128 lanes x 2 flops at 2.1 GHz x 2 (packed) could give."""
    r32 = B.gpe_fma_rate(0, 1 << 12)
    r64 = B.gpe_fma_rate(2, 1 << 8)
    r2 = B.gpe_fma_rate(1, 1 << 11)
    ceiling = 152 * 128 * 2 * 2.1e9 * 2
    for r in (r32, r64, r2):
        assert np.isfinite(r) and 0 < r < ceiling
    assert r32 > r64


@pytest.mark.parametrize("dtype,n,steps,tol", [("c128", 4096, 120, 1e-11), ("c128", 8192, 60, 1e-11),
                                               ("c128", 16384, 40, 1e-11), ("c64", 8192, 200, 1e-4),
                                               ("c64", 16384, 200, 1e-4), ("c64", 32768, 200, 1e-4)])
def test_cluster_1d(B, dtype, n, steps, tol):
    """1D grids held by a thread-block cluster (radix-C step across the blocks), FP32 at the
    200-step bar."""
    ntraj, dt, seed = 2, 0.02, 13
    b = B.GPEBatch((n,), ntraj, dtype, C0, C1, Q, dt)
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial((n,), ntraj, seed), dt, steps, 1)
    assert rel_l2_per_comp(gpu, ref) <= tol
    b.close()


def test_ragged_graph_replay(B):
    """Mixed shapes (cluster 1D, resident 1D, two 2D sizes) advanced with and without CUDA
    graph replay: bitwise identical, and equal to the oracle."""
    shapes = [(8192,), (1024,), (128, 128), (256, 256), (1024,), (128, 128)]
    outs = []
    for graph in (False, True):
        b = B.GPEBatch(list(shapes), dtype="c64", dt=0.02)
        b.set_graph(graph)
        b.init_noise(71, MEAN, 0.5)
        for _ in range(3):
            b.step(20)
        assert b.sync_status() == B.GPE_OK
        outs.append([p.cpu().clone() for p in b.psi])
        b.close()
    for a, c in zip(*outs):
        assert torch.equal(a, c)
    for i, s in enumerate(shapes):
        ref = run_oracle(oracle_initial(s, 1, 71, ids=[i]), 0.02, 60, len(s))
        assert rel_l2_per_comp(outs[1][i].numpy()[None].astype(np.complex128), ref) <= 1e-4


@pytest.mark.parametrize("dtype,shape,ntraj,steps,tol", [("c128", (256,), 2, 200, 1e-11), ("c128", (64, 128), 2, 100, 1e-11),
                                                          ("c128", (8192,), 1, 40, 1e-11), ("c64", (128, 128), 2, 200, 1e-4),
                                                          ("c128", (64, 64, 64), 1, 10, 1e-11)])
def test_rotation_integrator(B, dtype, shape, ntraj, steps, tol):
    """Spin-rotation local step against the oracle's rotation scheme; F_z conserved."""
    seed, dt = 21, 0.02
    b = B.GPEBatch(shape, ntraj, dtype, C0, C1, Q, dt)
    b.set_integrator(B.GPE_INTEGRATOR_ROTATION)
    b.init_noise(seed, MEAN, 0.5)
    psi0 = b.psi.cpu().numpy() if b.uniform else None
    b.step(steps)
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = O.propagate_rotation(torch.as_tensor(oracle_initial(shape, ntraj, seed)), dt, steps, C0, C1, Q, 1.0,
                               len(shape)).numpy()
    assert rel_l2_per_comp(gpu, ref) <= tol
    d = len(shape)
    ax = tuple(range(1, 1 + d))
    n0 = np.abs(psi0.astype(np.complex128)) ** 2
    n1 = np.abs(gpu) ** 2
    fz0 = (n0[:, 0] - n0[:, 2]).sum(axis=ax)
    fz1 = (n1[:, 0] - n1[:, 2]).sum(axis=ax)
    assert np.abs(fz1 - fz0).max() <= (1e-10 if dtype == "c128" else 1e-4) * np.abs(n0).sum()
    b.close()


def test_trajectory_base_draws_the_same_ensemble(B):
    """A batch with base 5 and 3 trajectories draws trajectories 5..7 of one large batch."""
    big = B.GPEBatch((64, 64), 8, "c64")
    big.init_noise(3, MEAN, 0.5)
    small = B.GPEBatch((64, 64), 3, "c64")
    small.set_traj_base(5)
    small.init_noise(3, MEAN, 0.5)
    torch.cuda.synchronize()
    assert torch.equal(big.psi[5:8], small.psi)
    big.close()
    small.close()


def test_full_size_3d_256_sampled(B):
    """3D 256^3 x 8 trajectories (3.2 GB of fields), the 3D workload's launch
    configuration; one trajectory checked against the oracle after 2 steps, and F_z / E
    drift logged through the diagnostics."""
    wl = W.C3_3D[1]
    b = B.GPEBatch(wl.shape, wl.ntraj, "c64", wl.c0, wl.c1, wl.q, wl.dt)
    b.init_noise(W.SEED_BASE, wl.mean_spinor(), wl.noise_per_mode)
    nb, sd = b.layout()
    acc = b.new_accumulator(2)
    b.observables(acc, B.GPE_OBS_DIAG, 0)
    b.step(2)
    b.observables(acc, B.GPE_OBS_DIAG, 1)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi[3:4].cpu().numpy().astype(np.complex128)
    ref = run_oracle(oracle_initial(wl.shape, 1, W.SEED_BASE, ids=[3]), wl.dt, 2, 3, q=wl.q)
    assert rel_l2_per_comp(gpu, ref) <= 1e-5
    a = acc.cpu().numpy()
    _, d0 = B.unpack_slot(a[:sd], nb, wl.ntraj)
    _, d1 = B.unpack_slot(a[sd:], nb, wl.ntraj)
    N0 = d0[:, :3].sum(1)
    assert np.abs(d1[:, :3].sum(1) - N0).max() < 1e-5 * N0.max()
    b.close()

@pytest.mark.parametrize("shape,ntraj", [((256, 256), 3), ((64, 64, 64), 2), ((256, 64, 128), 2)])
def test_every_tile_width_gives_the_same_bits(B, shape, ntraj):
    """Every built tile width of the strided passes, fixed through gpe_batch_set_tiles, gives
    the fields of the default widths bit for bit; widths that are not built are refused."""
    def cands(n):
        return (2, 4, 8) if n >= 256 else (4, 8, 16)
    ny = shape[-2]   # shapes are (z,) y, x
    combos = [(cy, 0) for cy in cands(ny)] if len(shape) == 2 else \
        [(cy, cz) for cy in cands(ny) for cz in cands(shape[-3])]
    out = {}
    for cy, cz in [(None, None)] + combos:
        b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, 0.02)
        b.set_autotune(False)
        if cy is not None:
            b.set_tiles(cy, cz)
            assert b.tiles(0)[:2] == (cy, cz)
        b.init_noise(5, MEAN, 0.5)
        b.step(6)
        assert b.sync_status() == B.GPE_OK
        out[(cy, cz)] = b.psi.cpu().numpy()
        if cy is None:
            with pytest.raises(B.GPEError):
                b.set_tiles(3)
            with pytest.raises(B.GPEError):
                b.set_tiles(cands(ny)[0], 4 if len(shape) == 2 else 32)
        b.close()
    ref = out.pop((None, None))
    for key, v in out.items():
        np.testing.assert_array_equal(v, ref, err_msg=f"tile widths {key}")



@pytest.mark.parametrize("shape,ntraj", [((256, 256), 4), ((64, 128, 64), 2), ((128, 1024), 2)])
def test_autotuned_tiles_change_no_bit(B, shape, ntraj):
    """The column-pass tile widths the autotuner picks are among the built candidates, and
    the fields are bitwise the same as with the fixed default widths."""
    out = []
    for tune in (False, True):
        b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, 0.02)
        b.set_autotune(tune)
        b.init_noise(21, MEAN, 0.5)
        b.step(7)
        b.step(5)
        assert b.sync_status() == B.GPE_OK
        cy, cz, tuned = b.tiles(0)
        assert tuned == tune
        assert cy in (2, 4, 8, 16) and (cz in (2, 4, 8, 16) if len(shape) == 3 else cz == 0)
        assert b.xpass_threads(0) in (128, 192, 256)
        out.append(b.psi.cpu().numpy())
        b.close()
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("shape,ntraj", [((64, 64), 3), ((128, 128), 2), ((256, 64, 128), 2), ((1024, 512), 1),
                                         ((512, 1024), 1), ((64, 512), 5), ((64, 64, 512), 1)])
def test_every_xpass_block_size_gives_the_same_bits(B, shape, ntraj):
    """Every x-pass block size (128 and 256 threads, and 192 at an x extent of 512; fixed
    through gpe_batch_set_xpass_threads; rows per block change, the per-row arithmetic does
    not) gives the same fields bit for bit; sizes that are not built and FP64 batches are
    refused."""
    out = []
    for th in ((128, 192, 256) if shape[-1] == 512 else (128, 256)):
        b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, 0.02)
        b.set_autotune(False)
        b.set_xpass_threads(th)
        assert b.xpass_threads(0) == th
        b.init_noise(9, MEAN, 0.5)
        b.step(5)
        assert b.sync_status() == B.GPE_OK
        out.append(b.psi.cpu().numpy())
        with pytest.raises(B.GPEError):
            b.set_xpass_threads(160)
        if shape[-1] != 512:
            with pytest.raises(B.GPEError):
                b.set_xpass_threads(192)
        b.close()
    for o in out[1:]:
        np.testing.assert_array_equal(o, out[0])
    b = B.GPEBatch(shape, 1, "c128")
    with pytest.raises(B.GPEError) as ei:
        b.set_xpass_threads(128)
    assert ei.value.status == B.GPE_EUNSUPPORTED
    b.close()


@pytest.mark.parametrize("graph", [False, True])
def test_trajectory_lanes_change_no_bit(B, graph):
    """Splitting each 2D/3D shape group into trajectory lanes on their own streams
    (gpe_batch_set_lanes) changes no result bit: a uniform 2D batch, a 3D batch, a ragged
    mix with a 1D group (always one lane) and a 2D group whose fields are not back to back
    (pointer tables instead of tensor maps), direct launches and graph replay."""
    cases = [((128, 128), 5), ((64, 64, 64), 3)]
    for shape, ntraj in cases:
        out = {}
        for lanes in (1, 2, 3, 64):
            b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, 0.02)
            b.set_graph(graph)
            assert b.lanes(0) == (2 if len(shape) == 2 else 1)   # the default
            b.set_lanes(lanes)
            assert b.lanes(0) == min(lanes, ntraj)
            b.init_noise(13, MEAN, 0.5)
            b.step(4)
            b.step(3)
            assert b.sync_status() == B.GPE_OK
            out[lanes] = b.psi.cpu().numpy()
            b.close()
        for lanes, v in out.items():
            np.testing.assert_array_equal(v, out[1], err_msg=f"{shape} lanes={lanes}")
    shapes = [(1024,), (128, 128), (1024,), (128, 128), (128, 128)]
    ragged = {}
    for lanes in (1, 2, -1):
        b = B.GPEBatch(list(shapes), dtype="c64", dt=0.02)
        b.set_graph(graph)
        b.set_lanes(lanes)
        assert b.lanes(0) == 1 and b.lanes(1) == (1 if lanes == -1 else lanes)
        b.init_noise(29, MEAN, 0.5)
        b.step(6)
        assert b.sync_status() == B.GPE_OK
        ragged[lanes] = [p.cpu().clone() for p in b.psi]
        b.close()
    for lanes, v in ragged.items():
        for a, c in zip(v, ragged[1]):
            assert torch.equal(a, c), f"ragged lanes={lanes}"
    # three 2D trajectories in separate allocations (not back to back)
    noncontig = {}
    for lanes in (1, 2, 3):
        fields = [torch.zeros((3, 128, 128), dtype=torch.complex64, device="cuda") for _ in range(3)]
        pad = [torch.zeros(64, device="cuda") for _ in range(3)]   # keep the allocations apart
        h = B.gpe_batch_create([((128, 128), 1.0, f) for f in fields], B.GPE_C64, C0, C1, Q, 0.02)
        try:
            B._check(B.LIB.gpe_batch_set_graph(h, 1 if graph else 0))
            B._check(B.LIB.gpe_batch_set_lanes(h, lanes))
            B.tw_init_noise(h, 31, MEAN, 0.5)
            B.gpe_step_batch(h, 5)
            assert B.gpe_sync_status(h) == B.GPE_OK
            noncontig[lanes] = [f.cpu().clone() for f in fields]
        finally:
            B.gpe_batch_destroy(h)
        del pad
    for lanes, v in noncontig.items():
        for a, c in zip(v, noncontig[1]):
            assert torch.equal(a, c), f"separate allocations lanes={lanes}"
    b = B.GPEBatch((64, 64), 2, "c64")
    for bad in (0, -2, 65):
        with pytest.raises(B.GPEError) as ei:
            b.set_lanes(bad)
        assert ei.value.status == B.GPE_EINVAL
    b.close()


def test_resident_4096_fp32_split_calls(B):
    """The paper's 1D grid in FP32 (resident kernel with its last-stage twiddles and
    full-step phases in tensor memory, the half-step phases of a call's first and last step
    read from the table): calls of 1, 2, 0 and 37 steps, and one call of 40, against the
    oracle's single run."""
    shape, ntraj, dt, seed = (4096,), 3, 0.02, 19
    outs = []
    for chunks in ((1, 2, 0, 37), (40,)):
        b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, dt)
        b.init_noise(seed, MEAN, 0.5)
        for n in chunks:
            b.step(n)
        assert b.sync_status() == B.GPE_OK
        outs.append(b.psi.cpu().numpy())
        b.close()
    ref = run_oracle(oracle_initial(shape, ntraj, seed), dt, 40, 1)
    assert rel_l2_per_comp(outs[0].astype(np.complex128), ref) <= 1e-4
    assert rel_l2_per_comp(outs[1].astype(np.complex128), ref) <= 1e-4


@pytest.mark.parametrize("shape,ntraj,steps", [((4096,), 3, 30), ((4096,), 2, 1), ((2048,), 5, 30), ((2048,), 1, 1),
                                               ((8192,), 2, 20), ((16384,), 1, 12), ((32768,), 1, 5)])
def test_table_memory_forms_give_the_same_bits(B, shape, ntraj, steps):
    """The 1D kernels that keep each thread's last-stage twiddles and full-step phases in
    tensor memory (resident at 4096 and 2048 points, cluster slices of 4096; FP32) give the fields of
    the form that reads them through L1 (gpe_debug_table_memory(0)) bit for bit."""
    outs = {}
    try:
        for mode in (1, 0):
            B._check(B.LIB.gpe_debug_table_memory(mode))
            b = B.GPEBatch(shape, ntraj, "c64", C0, C1, Q, 0.02)
            b.init_noise(23, MEAN, 0.5)
            b.step(steps)
            b.step(2)
            assert b.sync_status() == B.GPE_OK
            outs[mode] = b.psi.cpu().numpy()
            b.close()
    finally:
        B._check(B.LIB.gpe_debug_table_memory(1))
    np.testing.assert_array_equal(outs[1].view(np.uint32), outs[0].view(np.uint32))


def test_full_size_ragged_mix_sampled(B):
    """The ragged workload (200 1D trajectories of 1024-16384 points and 32 2D ones of
    128^2-1024^2, FP32) in the launch configuration the bench times (one batch, graph replay):
    after 50 steps, sampled trajectories of every kernel kind (cluster and resident 1D, 2D)
    equal, bit for bit, the same trajectory advanced alone (its noise reproduced through the
    trajectory base); a 128^2 one matches the oracle; every trajectory keeps its norm."""
    shapes = W.ragged_sizes()
    seed, steps = W.SEED_BASE, 50
    b = B.GPEBatch(list(shapes), dtype="c64", c0=1.0, c1=-0.1, q=0.09, dt=0.02)
    b.set_graph(True)
    b.init_noise(seed, MEAN, 0.5)
    n0 = [float((p.to(torch.complex128).abs() ** 2).sum()) for p in b.psi]
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    n1 = [float((p.to(torch.complex128).abs() ** 2).sum()) for p in b.psi]
    assert max(abs(a - c) / a for a, c in zip(n0, n1)) < 2e-5
    picks = {}
    for i, s in enumerate(shapes):
        kind = "cluster" if len(s) == 1 and s[0] > 4096 else ("resident" if len(s) == 1 else f"2d{s[0]}")
        picks.setdefault(kind, i)
    for kind, i in picks.items():
        s = shapes[i]
        solo = B.GPEBatch(s, 1, "c64", 1.0, -0.1, 0.09, 0.02)
        solo.set_traj_base(i)
        solo.init_noise(seed, MEAN, 0.5)
        solo.step(steps)
        assert solo.sync_status() == B.GPE_OK
        assert torch.equal(solo.psi[0], b.psi[i]), f"{kind} trajectory {i} {s}"
        solo.close()
    i = picks.get("2d128")
    if i is not None:
        ref = run_oracle(oracle_initial(shapes[i], 1, seed, ids=[i]), 0.02, steps, 2)
        assert rel_l2_per_comp(b.psi[i].cpu().numpy()[None].astype(np.complex128), ref) <= 1e-4
    b.close()


def test_full_config_1d_256_fp64_spectra_every_100(B):
    """The 1D workload at its full configuration: 256 points, FP64, one trajectory from the
    noisy polar state, dt = 0.01, 1000 steps, occupation spectra, S_perp and diagnostics
    every 100 steps (11 samples with t = 0), each sample against the oracle's run."""
    wl = W.C1_1D
    seed = W.SEED_BASE
    b = B.GPEBatch(wl.shape, wl.ntraj, wl.dtype, wl.c0, wl.c1, wl.q, wl.dt, dx=wl.dx)
    b.init_noise(seed, wl.mean_spinor(), wl.noise_per_mode)
    nb, sd = b.layout()
    nsamples = wl.steps // wl.sample_every + 1
    acc = b.new_accumulator(nsamples)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
    for i in range(1, nsamples):
        b.step(wl.sample_every)
        b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, i)
    assert b.sync_status() == B.GPE_OK
    a = acc.cpu().numpy().reshape(nsamples, sd)
    p = oracle_initial(wl.shape, 1, seed, npm=wl.noise_per_mode, mean=wl.mean_spinor())
    for i in range(nsamples):
        if i > 0:
            p = run_oracle(p, wl.dt, wl.sample_every, 1, c0=wl.c0, c1=wl.c1, q=wl.q, dx=wl.dx)
        spec, diag = B.unpack_slot(a[i], nb, 1)
        rs, rd, _ = oracle_observables(p, wl.dx, 1, q=wl.q)
        scale = np.abs(rs).max()
        assert np.abs(spec - rs).max() <= 1e-10 * scale, i
        np.testing.assert_allclose(diag, rd, rtol=1e-10, atol=1e-10 * np.abs(rd).max())
    b.close()


def test_host_upload_download_round_trip(B):
    """gpe_batch_upload / gpe_batch_download move every trajectory of the batch, in batch
    order and back to back, between host memory and the device fields (a uniform batch: one
    copy; a ragged one whose shape groups sit in separate allocations: several), and
    gpe_obs_download returns one accumulator slot."""
    for shapes in ([(64, 64)] * 3, [(256,), (64, 128), (256,), (64, 64, 64)]):
        b = B.GPEBatch(shapes[0], len(shapes), "c64") if len(set(shapes)) == 1 else \
            B.GPEBatch(list(shapes), dtype="c128")
        tdt = torch.complex64 if b.dtype == B.GPE_C64 else torch.complex128
        total = sum(3 * int(np.prod(s)) for s in shapes)
        g = torch.Generator().manual_seed(7)
        host = torch.complex(torch.randn(total, generator=g, dtype=torch.float64),
                             torch.randn(total, generator=g, dtype=torch.float64)).to(tdt).pin_memory()
        b.upload(host)
        torch.cuda.synchronize()
        dev = [b.psi[i] for i in range(len(shapes))] if b.uniform else b.psi
        flat = torch.cat([p.reshape(-1).cpu() for p in dev])
        assert torch.equal(flat, host)
        back = torch.zeros_like(host).pin_memory()
        b.download(back)
        torch.cuda.synchronize()
        assert torch.equal(back, host)
        b.close()
    b = B.GPEBatch((64, 64), 2, "c64")
    b.init_noise(3, MEAN, 0.5)
    nb, sd = b.layout()
    acc = b.new_accumulator(3)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 2)
    out = torch.zeros(sd, dtype=torch.float64).pin_memory()
    b.download_slot(acc, 2, out)
    torch.cuda.synchronize()
    assert torch.equal(out, acc[2 * sd:3 * sd].cpu())
    with pytest.raises(B.GPEError):
        B._check(B.LIB.gpe_obs_download(b.h, acc.data_ptr(), -1, out.data_ptr(), None))
    b.close()
