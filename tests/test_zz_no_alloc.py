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


def _host_diag(psi, dx, c0, c1, q):
    """The same real-space sums in float64 torch on the host (not the oracle: a plain
    restatement used only to check odd extents the batch API does not accept)."""
    p = psi.detach().cpu().to(torch.complex128)
    d = p.dim() - 2
    ax = tuple(range(2, 2 + d))
    n = p.real ** 2 + p.imag ** 2
    n1, n0, nm = n[:, 0], n[:, 1], n[:, 2]
    rho, fz = n1 + n0 + nm, n1 - nm
    fp = 2 ** 0.5 * (p[:, 0].conj() * p[:, 1] + p[:, 1].conj() * p[:, 2])
    vol = dx ** d
    sm = lambda x: x.sum(dim=tuple(a - 1 for a in ax)) * vol
    out = torch.zeros(p.shape[0], 8, dtype=torch.float64)
    out[:, 0], out[:, 1], out[:, 2] = sm(n1), sm(n0), sm(nm)
    out[:, 4] = q * sm(n1 + nm)
    out[:, 5] = 0.5 * c0 * sm(rho * rho)
    out[:, 6] = 0.5 * c1 * sm(fz * fz + fp.real ** 2 + fp.imag ** 2)
    return out.numpy()


@pytest.mark.parametrize("shape,ntraj", [((1000,), 3), ((3, 5, 7), 2), ((4097,), 1)])
def test_noalloc_odd_extents(B, shape, ntraj):
    """Extents that are not powers of two and a last site block that is only partly
    filled, checked against float64 sums on the host, twice in a row."""
    g = torch.Generator().manual_seed(7)
    psi = (torch.randn((ntraj, 3) + shape, generator=g, dtype=torch.float64)
           + 1j * torch.randn((ntraj, 3) + shape, generator=g, dtype=torch.float64)).to("cuda")
    ref = _host_diag(psi, 0.7, 1.0, -0.1, 0.09)
    for _ in range(2):
        out = torch.full((ntraj * 8,), float("nan"), dtype=torch.float64, device="cuda")
        B.gpe_diagnostics_noalloc(psi, len(shape), 1.0, -0.1, 0.09, 0.7, out)
        np.testing.assert_allclose(out.cpu().numpy().reshape(ntraj, 8), ref, rtol=1e-12, atol=1e-12)


def test_noalloc_at_capacity(B):
    """64 fields of 512^2 are exactly the 4096 site blocks the scratch holds: accepted,
    and equal to float64 host sums; one site block more is rejected."""
    import ctypes
    ntraj, shape = 64, (512, 512)
    g = torch.Generator().manual_seed(8)
    psi = (torch.randn((ntraj, 3) + shape, generator=g) + 1j * torch.randn((ntraj, 3) + shape, generator=g)).to(
        torch.complex64).to("cuda")
    out = torch.full((ntraj * 8,), float("nan"), dtype=torch.float64, device="cuda")
    B.gpe_diagnostics_noalloc(psi, 2, 1.0, -0.1, 0.09, 1.0, out)
    ref = _host_diag(psi, 1.0, 1.0, -0.1, 0.09)
    np.testing.assert_allclose(out.cpu().numpy().reshape(ntraj, 8), ref, rtol=1e-10, atol=1e-9)
    small = torch.zeros(16, dtype=torch.complex64, device="cuda")
    for dims, nt in (((512 * 512 + 1, 1, 1), 64), ((4096 * 4096 + 1, 1, 1), 1)):
        n = (ctypes.c_int32 * 3)(*dims)
        st = B.LIB.gpe_diagnostics_noalloc(ctypes.c_void_p(small.data_ptr()), nt, 1, n, 1.0, B.GPE_C64, 1.0, -0.1,
                                           0.09, ctypes.c_void_p(out.data_ptr()), None)
        assert st == B.GPE_EINVAL


def test_noalloc_rejects_overflowing_extents(B):
    """Three extents whose product wraps a 64-bit integer are rejected, not launched."""
    import ctypes
    small = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    big = 2 ** 31 - 1
    for dims in ((big, big, big), (big, big, 4), (1 << 22, 1 << 22, 1 << 22)):
        n = (ctypes.c_int32 * 3)(*dims)
        st = B.LIB.gpe_diagnostics_noalloc(ctypes.c_void_p(small.data_ptr()), 1, 3, n, 1.0, B.GPE_C64, 1.0, -0.1,
                                           0.09, ctypes.c_void_p(out.data_ptr()), None)
        assert st == B.GPE_EINVAL
        assert "capacity" in B.LIB.gpe_last_error().decode()
