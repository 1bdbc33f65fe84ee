"""Adjoint of the split step and the late-time S_perp loss on the GPU against the oracle's
autograd gradient (FP64) and central finite differences."""
import math

import numpy as np
import pytest
import torch

from oracle import gpe_oracle as O
from paper_2310_03636_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C0, C1 = 1.0, -0.1


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_03636_gb300 import binding
    return binding


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("shape,knots", [((64, 128), None), ((128, 64), [0.2, 0.1, 0.05]), ((128,), [0.3, 0.0]),
                                         ((64, 64, 64), None)])
def test_adjoint_step_matches_oracle_vjp(B, shape, knots):
    """One step's VJP: lam_n = J^T lam_{n+1} and dL/dq, L = Re sum conj(lam) psi_{n+1}."""
    d = len(shape)
    ntraj, dt, step = 2, 0.05, 3
    psi = W.random_field(shape, ntraj, seed=41, scale=0.7)
    lam = W.random_field(shape, ntraj, seed=42, scale=1.0, mean=(0.1, -0.2, 0.3))
    q0 = 0.09
    t_end = 10 * dt
    # oracle
    p = torch.as_tensor(psi).requires_grad_(True)
    if knots is None:
        qt = torch.tensor(q0, dtype=torch.float64, requires_grad=True)
        qn = qt
    else:
        qt = torch.tensor(knots, dtype=torch.float64, requires_grad=True)
        qn = O.q_piecewise_linear(qt, t_end)((step + 0.5) * dt)
    out = O.strang_step(p, dt, C0, C1, qn, 1.0, d)
    L = (torch.as_tensor(lam).conj() * out).real.sum()
    gp, gq = torch.autograd.grad(L, (p, qt))
    # GPU
    psi_d = torch.as_tensor(psi).cuda().contiguous()
    lam_d = torch.as_tensor(lam).cuda().contiguous()
    b = B.GPEBatch(shape, ntraj, "c128", C0, C1, q0, dt, q_knots=knots, t_end=t_end)
    dq = torch.zeros(len(knots) if knots else 1, dtype=torch.float64, device="cuda")
    B.gpe_adjoint_step(b.h, psi_d, lam_d, step, dq)
    assert b.sync_status() == B.GPE_OK
    assert rel(lam_d.cpu().numpy(), gp.numpy()) < 1e-11
    assert rel(dq.cpu().numpy(), np.atleast_1d(gq.numpy())) < 1e-10
    b.close()


def test_adjoint_step_fp32(B):
    shape, ntraj, dt = (64, 64), 2, 0.02
    psi = W.random_field(shape, ntraj, seed=5, scale=0.7)
    lam = W.random_field(shape, ntraj, seed=6, scale=1.0)
    p = torch.as_tensor(psi).requires_grad_(True)
    qt = torch.tensor(0.09, dtype=torch.float64, requires_grad=True)
    L = (torch.as_tensor(lam).conj() * O.strang_step(p, dt, C0, C1, qt, 1.0, 2)).real.sum()
    gp, gq = torch.autograd.grad(L, (p, qt))
    b = B.GPEBatch(shape, ntraj, "c64", C0, C1, 0.09, dt)
    psi_d = torch.as_tensor(psi).to(torch.complex64).cuda().contiguous()
    lam_d = torch.as_tensor(lam).to(torch.complex64).cuda().contiguous()
    dq = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.gpe_adjoint_step(b.h, psi_d, lam_d, 0, dq)
    assert rel(lam_d.cpu().numpy().astype(np.complex128), gp.numpy()) < 1e-5
    assert abs(float(dq[0]) - float(gq)) < 1e-4 * abs(float(gq))
    b.close()


@pytest.mark.parametrize("shape", [(64, 64), (256,), (64, 64, 64)])
def test_sf_band_loss_and_seed(B, shape):
    d = len(shape)
    dx, kmin, kmax = 1.0, 0.2, 0.4 if d > 1 else 0.6
    psi = W.random_field(shape, 3, seed=9, scale=0.8)
    p = torch.as_tensor(psi).requires_grad_(True)
    L = O.sf_band_loss(p, dx, d, kmin, kmax)
    (g,) = torch.autograd.grad(L, p)
    b = B.GPEBatch(shape, 3, "c128", C0, C1, 0.09, 0.02)
    psi_d = torch.as_tensor(psi).cuda().contiguous()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(psi_d)
    B.gpe_sf_band_loss(b.h, psi_d, kmin, kmax, loss, lam)
    assert abs(float(loss[0]) - float(L.detach())) < 1e-12 * abs(float(L.detach()))
    assert rel(lam.cpu().numpy(), g.numpy()) < 1e-11
    b.close()


def _oracle_loss(knots, psi0, shape, dt, nsteps, t_end, kmin, kmax):
    qf = O.q_piecewise_linear(knots, t_end)
    p = O.propagate(psi0, dt, nsteps, C0, C1, qf, 1.0, len(shape))
    return O.sf_band_loss(p, 1.0, len(shape), kmin, kmax)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-8), ("c64", 2e-3)])
def test_full_gradient_vs_oracle(B, dtype, tol):
    """SpinSFLoss through checkpoints (every 7 steps of 30) against oracle autograd."""
    from paper_2310_03636_gb300.adjoint import AdjointConfig, sf_loss
    shape, ntraj, dt, nsteps = (64, 64), 2, 0.05, 30
    knots = torch.tensor([0.2, 0.15, 0.08, 0.05], dtype=torch.float64)
    cfg = AdjointConfig(shape, nsteps, dt, t_end=nsteps * dt, kmin=0.3, kmax=1.1, c0=C0, c1=C1, dtype=dtype,
                        checkpoint_every=7)
    psi0 = torch.as_tensor(W.random_field(shape, ntraj, seed=3, scale=0.6))
    k1 = knots.clone().requires_grad_(True)
    p1 = psi0.clone().requires_grad_(True)
    Lo = _oracle_loss(k1, p1, shape, dt, nsteps, cfg.t_end, cfg.kmin, cfg.kmax)
    gk_o, gp_o = torch.autograd.grad(Lo, (k1, p1))
    k2 = knots.clone().requires_grad_(True)
    p2 = psi0.clone().cuda().requires_grad_(True)
    Lg = sf_loss(k2, p2, cfg)
    Lg.backward()
    Lo = float(Lo.detach())
    assert abs(float(Lg) - Lo) < max(tol, 1e-12) * abs(Lo) * (1 if dtype == "c128" else 10)
    assert rel(k2.grad.numpy(), gk_o.numpy()) < tol
    assert rel(p2.grad.cpu().numpy(), gp_o.numpy()) < tol


def test_gradient_vs_finite_differences(B):
    """FP64 GPU gradient w.r.t. two knots against central differences of the GPU forward."""
    from paper_2310_03636_gb300.adjoint import AdjointConfig, sf_loss
    shape, ntraj, dt, nsteps = (64, 64), 2, 0.02, 120
    knots = torch.tensor(W.q_ramp_knots(8), dtype=torch.float64)
    cfg = AdjointConfig(shape, nsteps, dt, t_end=nsteps * dt, kmin=0.2, kmax=0.4, dtype="c128",
                        checkpoint_every=32)
    psi0 = torch.as_tensor(W.random_field(shape, ntraj, seed=17, scale=0.5)).cuda()
    k = knots.clone().requires_grad_(True)
    L = sf_loss(k, psi0, cfg)
    L.backward()
    for j in (1, 5):
        h = 1e-5
        kp = knots.clone(); kp[j] += h
        km = knots.clone(); km[j] -= h
        fd = (float(sf_loss(kp, psi0, cfg)) - float(sf_loss(km, psi0, cfg))) / (2 * h)
        assert abs(fd - float(k.grad[j])) < 1e-5 * max(abs(fd), 1e-3)


def test_full_size_adjoint_workload(B):
    """2D 256^2 x 8 trajectories, 64-knot q ramp 0.2 -> 0.05, checkpoints every 256 steps.

    The gradient of the structure factor after the full 4096 steps (t = 82) is dominated
    by chaotic amplification of the tangent dynamics (~e^{0.4 t}), so no finite difference
    can resolve it; at this size the test checks (1) that the full-length gradient runs
    and is finite in FP32 and FP64, (2) the FP64 gradient against central differences at
    a 200-step horizon on the full grid, (3) the adjoint identity Re<lam, J v> =
    Re<J^T lam, v> of one full-size step with J v from a central difference."""
    from paper_2310_03636_gb300.adjoint import AdjointConfig, sf_loss
    wl = W.C5_ADJ
    knots = torch.tensor(W.q_ramp_knots(64), dtype=torch.float64)
    ntraj = wl.ntraj
    b = B.GPEBatch(wl.shape, ntraj, "c128", wl.c0, wl.c1, wl.q, wl.dt)
    b.init_noise(W.SEED_BASE + 5, wl.mean_spinor(), wl.noise_per_mode)
    psi0 = b.psi.clone()
    b.close()
    # (1) full length, both precisions
    for dtype in ("c128", "c64"):
        cfg = AdjointConfig(wl.shape, wl.steps, wl.dt, t_end=wl.steps * wl.dt, kmin=0.2, kmax=0.4, c0=wl.c0,
                            c1=wl.c1, dtype=dtype, checkpoint_every=256)
        k = knots.clone().requires_grad_(True)
        p = psi0.clone().requires_grad_(True)
        L = sf_loss(k, p, cfg)
        L.backward()
        assert math.isfinite(float(L))
        assert torch.isfinite(k.grad).all() and torch.isfinite(torch.view_as_real(p.grad)).all()
    # (2) short horizon on the full grid
    n_short = 200
    cfg = AdjointConfig(wl.shape, n_short, wl.dt, t_end=n_short * wl.dt, kmin=0.2, kmax=0.4, c0=wl.c0, c1=wl.c1,
                        dtype="c128", checkpoint_every=64)
    k = knots.clone().requires_grad_(True)
    L = sf_loss(k, psi0, cfg)
    L.backward()
    for j in (10, 50):
        h = 1e-4
        kp = knots.clone(); kp[j] += h
        km = knots.clone(); km[j] -= h
        fd = (float(sf_loss(kp, psi0, cfg)) - float(sf_loss(km, psi0, cfg))) / (2 * h)
        g = float(k.grad[j])
        assert abs(fd - g) < 1e-4 * max(abs(fd), abs(g)), (j, fd, g)
    # (3) adjoint identity for one full-size step
    g = torch.Generator(device="cuda").manual_seed(7)
    v = torch.randn(psi0.shape, dtype=torch.complex128, device="cuda", generator=g)
    lam = torch.randn(psi0.shape, dtype=torch.complex128, device="cuda", generator=g)
    hh = 1e-6
    bp = B.GPEBatch(wl.shape, ntraj, "c128", wl.c0, wl.c1, wl.q, wl.dt, psi=(psi0 + hh * v).contiguous())
    bp.step(1)
    bm = B.GPEBatch(wl.shape, ntraj, "c128", wl.c0, wl.c1, wl.q, wl.dt, psi=(psi0 - hh * v).contiguous())
    bm.step(1)
    jv = (bp.psi - bm.psi) / (2 * hh)
    lhs = float((lam.conj() * jv).real.sum())
    lam_in = lam.clone()
    dq = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.gpe_adjoint_step(bp.h, psi0.contiguous(), lam_in, 0, dq)
    rhs = float((lam_in.conj() * v).real.sum())
    assert abs(lhs - rhs) < 1e-7 * abs(lhs)
    bp.close()
    bm.close()


@pytest.mark.parametrize("dtype,shape,knots", [("c128", (64, 128), [0.2, 0.1, 0.05]), ("c64", (128, 128), None),
                                               ("c64", (64, 64, 64), [0.1, 0.3]), ("c128", (512,), [0.2, 0.05]),
                                               ("c64", (1024,), None)])
def test_adjoint_segment_equals_step_by_step(B, dtype, shape, knots):
    """gpe_adjoint_segment (recompute and reverse sweep of one checkpoint segment inside the
    library) against the step-by-step calls (recompute with gpe_step_batch(1), then
    gpe_adjoint_step per step): bit for bit in 1D, where it makes those calls; in 2D/3D, where
    it recomputes with merged kinetic half steps, equal to rounding (relative 1e-11 in FP64,
    1e-4 in FP32); the step counter ends at n0 + nseg - 1 either way."""
    ntraj, dt, n0, nseg = 2, 0.03, 5, 11
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    ck = torch.as_tensor(W.random_field(shape, ntraj, seed=51, scale=0.8)).to("cuda", tdt).contiguous()
    lam0 = torch.as_tensor(W.random_field(shape, ntraj, seed=52, scale=1.0)).to("cuda", tdt).contiguous()
    nk = len(knots) if knots else 1
    kw = dict(q_knots=knots, t_end=30 * dt) if knots else {}
    res = []
    for mode in ("loop", "segment"):
        psi = torch.zeros_like(ck)
        b = B.GPEBatch(shape, ntraj, dtype, C0, C1, 0.09, dt, psi=psi, **kw)
        b.set_autotune(False)
        lam = lam0.clone()
        dq = torch.zeros(nk, dtype=torch.float64, device="cuda")
        if mode == "loop":
            psi.copy_(ck)
            b.set_step(n0)
            states = [ck.clone()]
            for _ in range(nseg - 1):
                b.step(1)
                states.append(psi.clone())
            for j in range(nseg - 1, -1, -1):
                B.gpe_adjoint_step(b.h, states[j], lam, n0 + j, dq)
        else:
            ws = torch.empty((nseg,) + tuple(ck.shape), dtype=tdt, device="cuda")
            B.gpe_adjoint_segment(b.h, ck, ws, n0, nseg, lam, dq)
        assert b.sync_status() == B.GPE_OK
        res.append((lam.cpu().numpy(), dq.cpu().numpy(), b.step_count))
        b.close()
    (l1, q1, s1), (l2, q2, s2) = res
    assert s1 == s2 == n0 + nseg - 1
    if len(shape) == 1:
        np.testing.assert_array_equal(l1, l2)
        np.testing.assert_array_equal(q1, q2)
    else:
        tol = 1e-11 if dtype == "c128" else 1e-4
        assert rel(l2, l1) <= tol
        assert rel(q2, q1) <= tol
    b = B.GPEBatch(shape, ntraj, dtype, C0, C1, 0.09, dt)
    ws = torch.empty((1,) + tuple(ck.shape), dtype=tdt, device="cuda")
    dq = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.GPEError) as ei:
        B._check(B.LIB.gpe_adjoint_segment(b.h, ck.data_ptr(), ws.data_ptr(), 0, 0, lam0.data_ptr(),
                                           dq.data_ptr(), None))
    assert ei.value.status == B.GPE_EINVAL
    b.close()
