"""External potential V_m(x) in the diagonal step and non-uniform initial mean fields on the
GPU, against the FP64 oracle on the same seeded inputs (tolerances as in the propagation
parity tests: 1e-11 for FP64 fields, 1e-4 for FP32 fields)."""
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


def initial(shape, ntraj, seed, field=None):
    out = []
    for t in range(ntraj):
        eta = tw_noise(shape, seed, t, 0.5, 1.0)
        for m in range(3):
            eta[m] += MEAN[2 * m] + 1j * MEAN[2 * m + 1]
        if field is not None:
            eta = eta + field
        out.append(eta)
    return np.stack(out)


def rel_l2_per_comp(gpu, ref):
    ax = tuple(range(2, gpu.ndim))
    num = np.sqrt((np.abs(gpu - ref) ** 2).sum(axis=ax))
    den = np.sqrt((np.abs(ref) ** 2).sum(axis=ax))
    return float((num / den).max())


@pytest.mark.parametrize("dtype,shape,ntraj,steps,tol,rotation", [
    ("c128", (64, 128), 2, 100, 1e-11, False),
    ("c64", (128, 128), 2, 200, 1e-4, False),
    ("c128", (256,), 2, 200, 1e-11, False),        # resident 1D kernel
    ("c128", (4096,), 1, 60, 1e-11, False),        # cluster 1D kernel (FP64)
    ("c64", (8192,), 1, 100, 1e-4, False),         # cluster 1D kernel (FP32)
    ("c128", (64, 64, 64), 1, 10, 1e-11, False),
    ("c128", (64, 128), 2, 100, 1e-11, True),
    ("c64", (256,), 2, 200, 1e-4, True),
])
def test_potential_propagation(B, dtype, shape, ntraj, steps, tol, rotation):
    seed, dt = 777, 0.02
    V = W.smooth_potential(shape, seed=31, amp=0.3)
    b = B.GPEBatch(shape, ntraj, dtype, C0, C1, Q, dt)
    if rotation:
        b.set_integrator(B.GPE_INTEGRATOR_ROTATION)
    b.set_potential(torch.as_tensor(V))
    b.init_noise(seed, MEAN, 0.5)
    b.step(steps)
    assert b.sync_status() == B.GPE_OK
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    psi0 = torch.as_tensor(initial(shape, ntraj, seed))
    prop = O.propagate_rotation if rotation else O.propagate
    ref = prop(psi0, dt, steps, C0, C1, Q, 1.0, len(shape), V=V).numpy()
    assert rel_l2_per_comp(gpu, ref) <= tol
    # the potential matters at this size: without it the result is far away
    free = prop(psi0, dt, steps, C0, C1, Q, 1.0, len(shape)).numpy()
    assert rel_l2_per_comp(free, ref) > 100 * tol
    b.close()


def test_potential_energy_in_diagnostics(B):
    shape, ntraj, dx = (128, 64), 2, 0.8
    V = W.smooth_potential(shape, seed=2, amp=0.4, dx=dx)
    b = B.GPEBatch(shape, ntraj, "c128", C0, C1, Q, 0.02, dx=dx)
    b.set_potential(torch.as_tensor(V))
    b.init_noise(5, MEAN, 0.5)
    b.step(20)
    nb, sd = b.layout()
    acc = b.new_accumulator(1)
    b.observables(acc, B.GPE_OBS_DIAG, 0)
    assert b.sync_status() == B.GPE_OK
    _, diag = B.unpack_slot(acc, nb, ntraj)
    ref = O.diagnostics(torch.as_tensor(b.psi.cpu().numpy()), dx, C0, C1, Q, 2, V=V).numpy()
    np.testing.assert_allclose(diag, ref, rtol=1e-10, atol=1e-9)
    assert np.all(np.abs(diag[:, 7]) > 1.0)
    # removing the potential zeroes E_V
    b.set_potential(None)
    acc.zero_()
    b.observables(acc, B.GPE_OBS_DIAG, 0)
    _, diag = B.unpack_slot(acc, nb, ntraj)
    assert np.all(diag[:, 7] == 0.0)
    b.close()


def test_potential_invalidates_step_graphs(B):
    """A graph captured before the potential was set must not be replayed after it."""
    shape, ntraj, dt = (64, 64), 2, 0.02
    V = W.smooth_potential(shape, seed=7, amp=0.5)
    b = B.GPEBatch(shape, ntraj, "c128", C0, C1, Q, dt)
    b.set_graph(True)
    b.init_noise(3, MEAN, 0.5)
    b.step(15)
    b.set_potential(torch.as_tensor(V))
    b.init_noise(3, MEAN, 0.5)
    b.step(15)
    assert b.sync_status() == B.GPE_OK
    ref = O.propagate(torch.as_tensor(initial(shape, ntraj, 3)), dt, 15, C0, C1, Q, 1.0, 2, V=V).numpy()
    assert rel_l2_per_comp(b.psi.cpu().numpy(), ref) <= 1e-11
    b.close()


def test_potential_adjoint_step(B):
    """VJP of one step with a potential against the oracle's autograd."""
    shape, ntraj, dt, step = (64, 128), 2, 0.05, 2
    V = W.smooth_potential(shape, seed=13, amp=0.6)
    psi = W.random_field(shape, ntraj, seed=41, scale=0.7)
    lam = W.random_field(shape, ntraj, seed=42, scale=1.0, mean=(0.1, -0.2, 0.3))
    p = torch.as_tensor(psi).requires_grad_(True)
    qt = torch.tensor(Q, dtype=torch.float64, requires_grad=True)
    out = O.strang_step(p, dt, C0, C1, qt, 1.0, 2, V=V)
    L = (torch.as_tensor(lam).conj() * out).real.sum()
    gp, gq = torch.autograd.grad(L, (p, qt))
    b = B.GPEBatch(shape, ntraj, "c128", C0, C1, Q, dt)
    b.set_potential(torch.as_tensor(V))
    psi_d = torch.as_tensor(psi).cuda().contiguous()
    lam_d = torch.as_tensor(lam).cuda().contiguous()
    dq = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.gpe_adjoint_step(b.h, psi_d, lam_d, step, dq)
    assert b.sync_status() == B.GPE_OK
    g = gp.numpy()
    assert np.linalg.norm((lam_d.cpu().numpy() - g).ravel()) <= 1e-11 * np.linalg.norm(g.ravel())
    assert abs(float(dq[0]) - float(gq)) <= 1e-10 * abs(float(gq))
    b.close()


@pytest.mark.parametrize("dtype,shape", [("c128", (64, 64)), ("c64", (256,))])
def test_mean_field_initial_state(B, dtype, shape):
    """psi = mean spinor + mean field + the same noise as without a mean field."""
    field = W.smooth_random_field(shape, 1, seed=19, mean=(0.3, -0.1, 0.2))[0]
    b = B.GPEBatch(shape, 2, dtype)
    b.set_mean_field(torch.as_tensor(field))
    b.init_noise(99, MEAN, 0.5)
    gpu = b.psi.cpu().numpy().astype(np.complex128)
    ref = initial(shape, 2, 99, field)
    tol = 1e-13 if dtype == "c128" else 2e-7
    assert np.abs(gpu - ref).max() <= tol * np.abs(ref).max()
    b.set_mean_field(None)
    b.init_noise(99, MEAN, 0.5)
    np.testing.assert_allclose(b.psi.cpu().numpy().astype(np.complex128), initial(shape, 2, 99),
                               atol=tol * np.abs(ref).max())
    b.close()


def test_potential_argument_errors(B):
    b = B.GPEBatch((64, 64), 1, "c128")
    with pytest.raises(B.GPEError) as ei:
        B.gpe_batch_set_potential(b.h, (32, 64), torch.zeros((3, 32, 64), dtype=torch.float64, device="cuda"))
    assert ei.value.status == B.GPE_EINVAL
    with pytest.raises(B.GPEError) as ei:
        B.gpe_batch_set_mean_field(b.h, (64, 32), torch.zeros((3, 64, 32), dtype=torch.complex128, device="cuda"))
    assert ei.value.status == B.GPE_EINVAL
    b.close()
