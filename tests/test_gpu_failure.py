"""Failure paths, reached without faulting the GPU: bounded waits made to expire by a test
setting (a first-wait poll limit of zero), and device allocations made to fail on the host
by a test hook.  The library must report GPE_ETIMEOUT / GPE_ENOMEM, leave the context
usable and work normally afterwards."""
import numpy as np
import pytest
import torch

from oracle import gpe_oracle as O
from oracle.philox import tw_noise

pytestmark = pytest.mark.gpu

MEAN = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_03636_gb300 import binding
    yield binding
    binding.LIB.gpe_debug_fail_alloc(-1)


def _oracle(shape, ntraj, seed, steps, dt=0.02):
    psi = []
    for t in range(ntraj):
        eta = tw_noise(shape, seed, t, 0.5, 1.0)
        eta[1] += 1.0
        psi.append(eta)
    return O.propagate(torch.as_tensor(np.stack(psi)), dt, steps, 1.0, -0.1, 0.09, 1.0, len(shape)).numpy()


def _rel(gpu, ref):
    d = gpu.ndim - 2
    ax = tuple(range(2, 2 + d))
    return float((np.sqrt((abs(gpu - ref) ** 2).sum(axis=ax)) / np.sqrt((abs(ref) ** 2).sum(axis=ax))).max())


@pytest.mark.parametrize("dtype,shape", [("c64", (256, 256)), ("c64", (64, 64, 128)), ("c128", (128, 64))])
def test_expired_wait_reports_timeout_and_recovers(B, dtype, shape):
    """First copy waits limited to zero polls: every x-pass and tensor-map strided-pass block
    records GPE_ETIMEOUT, waits for its copies and returns without writing, so the fields
    are unchanged; with the default limit restored the batch steps cleanly again."""
    ntraj, seed = 2, 31
    b = B.GPEBatch(shape, ntraj, dtype, 1.0, -0.1, 0.09, 0.02)
    b.set_autotune(False)
    if dtype == "c64":
        assert b.tiles(0)[0] != 0     # contiguous batch: the tensor-map strided pass runs
    b.init_noise(seed, MEAN, 0.5)
    before = b.psi.clone()
    b.set_wait_limit(0)
    b.step(1)
    assert b.sync_status() == B.GPE_ETIMEOUT
    assert torch.equal(b.psi, before)
    assert b.sync_status() == B.GPE_OK          # the status word was cleared by the read
    b.set_wait_limit(-1)
    b.set_step(0)
    b.step(20)
    assert b.sync_status() == B.GPE_OK
    ref = _oracle(shape, ntraj, seed, 20)
    tol = 1e-4 if dtype == "c64" else 1e-11
    assert _rel(b.psi.cpu().numpy().astype(np.complex128), ref) <= tol
    with pytest.raises(B.GPEError):
        b.set_wait_limit(-2)
    b.close()


def test_expired_wait_in_graph_mode(B):
    """The wait limit is a kernel argument: changing it drops captured graphs, so a replay
    picks up the new limit and the old one again."""
    b = B.GPEBatch((128, 128), 2, "c64", 1.0, -0.1, 0.09, 0.02)
    b.set_graph(True)
    b.init_noise(3, MEAN, 0.5)
    b.step(4)
    assert b.sync_status() == B.GPE_OK
    b.set_wait_limit(0)
    b.step(4)
    assert b.sync_status() == B.GPE_ETIMEOUT
    b.set_wait_limit(-1)
    b.step(4)
    assert b.sync_status() == B.GPE_OK
    b.close()


def test_forced_allocation_failure_in_create(B):
    """Each device allocation of gpe_batch_create made to fail in turn: the call returns
    GPE_ENOMEM and cleans up; once the hook is past the last allocation the batch works."""
    shape = (128, 128)
    failures = 0
    for k in range(64):
        B.LIB.gpe_debug_fail_alloc(k)
        try:
            b = B.GPEBatch(shape, 2, "c64", 1.0, -0.1, 0.09, 0.02)
        except B.GPEError as e:
            assert e.status == B.GPE_ENOMEM, e
            assert "cudaMalloc" in str(e) or "bin tables" in str(e)
            failures += 1
            continue
        B.LIB.gpe_debug_fail_alloc(-1)
        b.init_noise(1, MEAN, 0.5)
        b.step(3)
        assert b.sync_status() == B.GPE_OK
        b.close()
        break
    else:
        pytest.fail("the batch never got past its allocations")
    assert failures >= 5          # status word, pointer tables, phase and twiddle tables, bins


def test_forced_allocation_failure_in_observables_and_loss(B):
    """The observables workspace (allocated on first use) and the loss workspace fail
    cleanly with GPE_ENOMEM; the next call allocates them and succeeds."""
    b = B.GPEBatch((128, 128), 2, "c64", 1.0, -0.1, 0.09, 0.02)
    b.set_autotune(False)
    b.init_noise(4, MEAN, 0.5)
    b.step(2)
    acc = b.new_accumulator(1)
    for k in (0, 1, 2, 3):          # the first, second, third and fourth workspace buffer
        B.LIB.gpe_debug_fail_alloc(k)
        with pytest.raises(B.GPEError) as ei:
            b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
        assert ei.value.status == B.GPE_ENOMEM
    B.LIB.gpe_debug_fail_alloc(-1)
    b.observables(acc, B.GPE_OBS_SPECTRA | B.GPE_OBS_DIAG, 0)
    assert b.sync_status() == B.GPE_OK
    assert torch.isfinite(acc).all() and float(acc.abs().sum()) > 0
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.LIB.gpe_debug_fail_alloc(0)
    with pytest.raises(B.GPEError) as ei:
        B.gpe_sf_band_loss(b.h, b.psi, 0.2, 0.4, loss)
    assert ei.value.status == B.GPE_ENOMEM
    B.LIB.gpe_debug_fail_alloc(-1)
    B.gpe_sf_band_loss(b.h, b.psi, 0.2, 0.4, loss)
    assert b.sync_status() == B.GPE_OK and float(loss) > 0
    b.close()
