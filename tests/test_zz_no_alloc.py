"""The allocation-free diagnostics entry point agrees with the batch API.

gpe_diagnostics_noalloc exists for callers that cannot let the library allocate device
memory (code that must not synchronise the device, processes whose device memory is all
owned by another allocator, health checks on a device that is out of memory).  It keeps
its partial sums in a fixed array compiled into the library.  This file is collected
last so that a failure here does not hide the other tests in a run that stops early.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MEAN = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_03636_gb300 import binding
    return binding


@pytest.mark.parametrize("dtype,shape,ntraj,dx,tol", [
    ("c128", (128, 128), 3, 0.8, 1e-10),
    ("c64", (512, 512), 5, 1.0, 1e-6),      # the batch API sums FP32 fields' terms in FP32 per thread
    ("c128", (2048,), 2, 0.5, 1e-10),
])
def test_noalloc_matches_observables(B, dtype, shape, ntraj, dx, tol):
    c0, c1, q = 1.0, -0.1, 0.09
    b = B.GPEBatch(shape, ntraj, dtype, c0, c1, q, 0.02, dx=dx)
    b.init_noise(99, MEAN, 0.5)
    b.step(10)
    nb, sd = b.layout()
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_DIAG, 0)
    ref = acc[4 * nb:4 * nb + 8 * ntraj].cpu().numpy().reshape(ntraj, 8)
    cols = [0, 1, 2, 4, 5, 6]
    for _ in range(2):        # two calls in a row: the shared scratch keeps no stale sums
        out = torch.full((ntraj * 8,), float("nan"), dtype=torch.float64, device="cuda")
        B.gpe_diagnostics_noalloc(b.psi, len(shape), c0, c1, q, dx, out)
        got = out.cpu().numpy().reshape(ntraj, 8)
        np.testing.assert_allclose(got[:, cols], ref[:, cols], rtol=tol, atol=tol * np.abs(ref[:, cols]).max())
        assert np.all(got[:, 3] == 0) and np.all(got[:, 7] == 0)
    b.close()


def test_noalloc_rejects_sizes_beyond_capacity(B):
    """2 fields of 4096 x 64 x 64 sites need 2 x 4096 site blocks: rejected before any
    device work (so a small buffer is enough to make the call)."""
    import ctypes
    psi = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    n = (ctypes.c_int32 * 3)(4096, 64, 64)
    st = B.LIB.gpe_diagnostics_noalloc(ctypes.c_void_p(psi.data_ptr()), 2, 3, n, 1.0, B.GPE_C64, 1.0, -0.1,
                                       0.09, ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.GPE_EINVAL
    assert "capacity" in B.LIB.gpe_last_error().decode()
