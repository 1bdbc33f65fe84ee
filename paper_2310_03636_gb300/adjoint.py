"""Gradients of a late-time spin structure factor with respect to a q(t) ramp and the
initial fields, through the library's hand-written adjoint (gpe_adjoint_step) with
checkpoint recomputation.  Marshalling and bookkeeping only: the forward steps, the loss,
its seed gradient and every adjoint step run in the library's kernels.
"""
from dataclasses import dataclass

import torch

from . import binding as B


@dataclass(frozen=True)
class AdjointConfig:
    shape: tuple            # spatial shape, slowest axis first
    nsteps: int
    dt: float
    t_end: float            # the q knots span [0, t_end]
    kmin: float
    kmax: float
    c0: float = 1.0
    c1: float = -0.1
    dx: float = 1.0
    dtype: str = "c64"
    checkpoint_every: int = 256


class SpinSFLoss(torch.autograd.Function):
    """loss(q_knots, psi0) = mean over trajectories of sum_{kmin <= |k| <= kmax} S_perp(k, T)
    after cfg.nsteps Strang steps from psi0 with q(t) piecewise linear through q_knots."""

    @staticmethod
    def forward(ctx, q_knots, psi0, cfg):
        knots = [float(x) for x in q_knots.detach().cpu().double().tolist()]
        ntraj = psi0.shape[0]
        tdt = torch.complex64 if cfg.dtype == "c64" else torch.complex128
        psi = psi0.detach().to(device="cuda", dtype=tdt).contiguous().clone()
        b = B.GPEBatch(cfg.shape, ntraj, cfg.dtype, cfg.c0, cfg.c1, knots[0], cfg.dt, dx=cfg.dx,
                       q_knots=knots, t_end=cfg.t_end, psi=psi)
        ckpts = []
        n = 0
        while n < cfg.nsteps:
            ckpts.append((n, psi.clone()))
            k = min(cfg.checkpoint_every, cfg.nsteps - n)
            b.step(k)
            n += k
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        B.gpe_sf_band_loss(b.h, psi, cfg.kmin, cfg.kmax, loss)
        ctx.b, ctx.ckpts, ctx.cfg, ctx.nknots = b, ckpts, cfg, len(knots)
        ctx.knot_dtype, ctx.knot_device = q_knots.dtype, q_knots.device
        ctx.psi_dtype, ctx.psi_device = psi0.dtype, psi0.device
        return loss[0].clone()

    @staticmethod
    def backward(ctx, g_loss):
        b, cfg = ctx.b, ctx.cfg
        psi = b.psi
        lam = torch.empty_like(psi)
        tmp = torch.zeros(1, dtype=torch.float64, device="cuda")
        B.gpe_sf_band_loss(b.h, psi, cfg.kmin, cfg.kmax, tmp, lam)
        lam.mul_(g_loss.to(device="cuda", dtype=torch.float64).item())
        dq = torch.zeros(max(1, ctx.nknots), dtype=torch.float64, device="cuda")
        bounds = [n for n, _ in ctx.ckpts] + [cfg.nsteps]
        states = torch.empty((cfg.checkpoint_every,) + tuple(psi.shape), dtype=psi.dtype, device=psi.device)
        for seg in range(len(ctx.ckpts) - 1, -1, -1):
            n0, ck = ctx.ckpts[seg]
            B.gpe_adjoint_segment(b.h, ck, states, n0, bounds[seg + 1] - n0, lam, dq)
        st = b.sync_status()
        if st != B.GPE_OK:
            raise B.GPEError(st, "device status after the adjoint sweep")
        b.close()
        grad_q = dq[:ctx.nknots].to(device=ctx.knot_device, dtype=ctx.knot_dtype)
        grad_psi = lam.to(device=ctx.psi_device, dtype=ctx.psi_dtype)
        return grad_q, grad_psi, None


def sf_loss(q_knots, psi0, cfg):
    return SpinSFLoss.apply(q_knots, psi0, cfg)
