"""Plain FP64 CPU oracle for the spin-1 Gross-Pitaevskii split-step hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` import this module.  The CUDA library and
its Python binding never import, call or link it, and it shares no code with them.

Written in plain PyTorch CPU ops on complex128 / float64 so that the same forward also
yields the exact gradient through autograd (used as the adjoint oracle).  Every step is
the plain definition: full d-dimensional FFTs, no merging of half kinetic steps, no
per-axis splitting, no fusion.

Paper: "Universal Dynamics at the Lowest Temperatures", Sec. 2.2.
  * Eq. (GPE): the three-component equation of motion, fields ordered (psi_1, psi_0, psi_-1).
  * The three split-step equations that follow Eq. (GPE): kinetic step in momentum space,
    diagonal phase step, off-diagonal (spin-mixing) 3x3 matrix step with predictor.
  * Sec. 2.1: structure factor S(t,k) = <F_perp(t,k)^* F_perp(t,k)>.

Readings of the paper used here (it is silent or garbled on these points):
  R1  predictor: psi~ = psi - i c1 dt S(psi) psi, and a~ = conj(psi~_-1) psi~_0,
      b~ = conj(psi~_0) psi~_1 (the printed definitions lack c1 dt and a conjugate);
  R2  the printed "ab cos(.) - 1" entries read ab (cos(.) - 1) and a*b* (cos(.) - 1);
  R3  lambda = 0 gives the identity matrix (the printed form is 0/0 there);
  R4  the diagonal step uses the densities of the field it acts on; it leaves them
      unchanged, so it is exact;
  R5  the printed order kinetic -> diagonal -> off-diagonal is symmetrised (Strang):
      K(dt/2) D(dt/2) O(dt) D(dt/2) K(dt/2), with q taken at the step midpoint;
  R6  hbar = m = 1; the potential V_m(x) of the diagonal step is optional (default 0,
      the homogeneous periodic box), one real field per component, the same for every
      trajectory, entering the diagonal step as V_m + f_m;
  R7  normalisations of n_m(k) and S_perp(k), radial bins b = round(|k| / (2 pi / L)).
"""
import math

import torch

CDT = torch.complex128
RDT = torch.float64


def _dims(d):
    return tuple(range(-d, 0))


def wavenumbers(n, dx):
    """k_j = 2 pi j / (n dx), j folded into [-n/2, n/2) (only k^2 and |k| are used)."""
    return 2.0 * math.pi * torch.fft.fftfreq(n, d=dx, dtype=RDT)


def k_squared(shape, dx):
    """|k|^2 on the grid of ``shape`` (spatial, slowest axis first)."""
    d = len(shape)
    k2 = torch.zeros(shape, dtype=RDT)
    for ax, n in enumerate(shape):
        k = wavenumbers(n, dx)
        view = [1] * d
        view[ax] = n
        k2 = k2 + (k * k).reshape(view)
    return k2


def _spatial_shape(psi, d):
    return tuple(psi.shape[-d:])


def kinetic(psi, tau, dx, d):
    """Kinetic part over a time tau: psi' = F^-1{ exp(-i tau |k|^2 / 2) F[psi] }.

    First split-step equation of Sec. 2.2 (hbar = m = 1), full d-dimensional FFT.
    psi: (..., 3, *shape) with d spatial axes.
    """
    shape = _spatial_shape(psi, d)
    phase = torch.exp(-0.5j * tau * k_squared(shape, dx))
    return torch.fft.ifftn(torch.fft.fftn(psi, dim=_dims(d)) * phase, dim=_dims(d))


def diag_phases(psi, c0, c1, q, d, V=None):
    """V_m + f_m: the diagonal entries of the operator in square brackets of Eq. (GPE).

    f_1  = q + (c0 + c1) rho + c1 (-2 |psi_-1|^2)
    f_0  = q + (c0 + c1) rho + c1 (-|psi_0|^2 - q / c1) = (c0 + c1) rho - c1 |psi_0|^2
    f_-1 = q + (c0 + c1) rho + c1 (-2 |psi_1|^2)
    (the -q/c1 entry cancels q for m = 0; written without the division so c1 = 0 works).
    V: optional real potential of shape (3, *shape), V_m(x) as in the diagonal step of
    Sec. 2.2 (None: V = 0).
    """
    n = psi.real ** 2 + psi.imag ** 2
    n1, n0, nm = n.select(-d - 1, 0), n.select(-d - 1, 1), n.select(-d - 1, 2)
    rho = n1 + n0 + nm
    f1 = q + (c0 + c1) * rho - 2.0 * c1 * nm
    f0 = (c0 + c1) * rho - c1 * n0
    fm = q + (c0 + c1) * rho - 2.0 * c1 * n1
    f = torch.stack([f1, f0, fm], dim=-d - 1)
    return f if V is None else f + torch.as_tensor(V, dtype=RDT)


def diag_step(psi, tau, c0, c1, q, d, V=None):
    """Diagonal part: psi'' = exp{-i [V_m + f_m] tau} psi' (second equation, Sec. 2.2)."""
    return psi * torch.exp(-1j * tau * diag_phases(psi, c0, c1, q, d, V))


def offdiag_matrix(a, b, theta_over_lambda, lam2):
    """The 3x3 matrix of the third split-step equation of Sec. 2.2, entry by entry.

    Written as printed with readings R2/R3: prefactor 1/lambda^2, angle lambda c1 dt.
    ``theta_over_lambda`` = c1 dt, ``lam2`` = |a|^2 + |b|^2.  Returns the nine entries
    U[i][j] (rows/cols ordered m = 1, 0, -1).
    """
    zero = lam2 == 0
    lam2s = torch.where(zero, torch.ones_like(lam2), lam2)
    lam = torch.sqrt(lam2s)
    th = lam * theta_over_lambda
    c, s = torch.cos(th), torch.sin(th)
    aa = a.real ** 2 + a.imag ** 2
    bb = b.real ** 2 + b.imag ** 2
    inv = 1.0 / lam2s
    u11 = (aa * c + bb) * inv
    u10 = -1j * a * lam * s * inv
    u1m = a * b * (c - 1.0) * inv
    u01 = -1j * a.conj() * lam * s * inv
    u00 = lam2s * c * inv
    u0m = -1j * b * lam * s * inv
    um1 = a.conj() * b.conj() * (c - 1.0) * inv
    um0 = -1j * b.conj() * lam * s * inv
    umm = (aa + bb * c) * inv
    one = torch.ones_like(u11)
    zc = torch.zeros_like(u10)
    u11 = torch.where(zero, one, u11)
    u00 = torch.where(zero, one, u00)
    umm = torch.where(zero, one, umm)
    u10 = torch.where(zero, zc, u10)
    u1m = torch.where(zero, zc, u1m)
    u01 = torch.where(zero, zc, u01)
    u0m = torch.where(zero, zc, u0m)
    um1 = torch.where(zero, zc, um1)
    um0 = torch.where(zero, zc, um0)
    return ((u11, u10, u1m), (u01, u00, u0m), (um1, um0, umm))


def spin_mixing_S_apply(a, b, p1, p0, pm):
    """S psi for S = off-diagonal part of the matrix in Eq. (GPE):
    S = [[0, a, 0], [a*, 0, b], [0, b*, 0]] with a = psi_-1^* psi_0, b = psi_0^* psi_1."""
    return a * p0, a.conj() * p1 + b * pm, b.conj() * p0


def offdiag_step(psi, tau, c1, d):
    """Off-diagonal interaction (spin-mixing) part over a time tau (third equation, Sec. 2.2).

    a and b are the averages of their values on psi and on the predictor
    psi~ = psi - i c1 tau S(psi) psi (reading R1); then psi <- U(a, b) psi.
    """
    p1, p0, pm = psi.select(-d - 1, 0), psi.select(-d - 1, 1), psi.select(-d - 1, 2)
    a0 = pm.conj() * p0
    b0 = p0.conj() * p1
    s1, s0, sm = spin_mixing_S_apply(a0, b0, p1, p0, pm)
    eps = c1 * tau
    t1 = p1 - 1j * eps * s1
    t0 = p0 - 1j * eps * s0
    tm = pm - 1j * eps * sm
    a = 0.5 * (a0 + tm.conj() * t0)
    b = 0.5 * (b0 + t0.conj() * t1)
    lam2 = a.real ** 2 + a.imag ** 2 + b.real ** 2 + b.imag ** 2
    U = offdiag_matrix(a, b, c1 * tau, lam2)
    n1 = U[0][0] * p1 + U[0][1] * p0 + U[0][2] * pm
    n0 = U[1][0] * p1 + U[1][1] * p0 + U[1][2] * pm
    nm = U[2][0] * p1 + U[2][1] * p0 + U[2][2] * pm
    return torch.stack([n1, n0, nm], dim=-d - 1)


def strang_step(psi, dt, c0, c1, q, dx, d, V=None):
    """One time step: K(dt/2) D(dt/2) O(dt) D(dt/2) K(dt/2) (reading R5)."""
    psi = kinetic(psi, 0.5 * dt, dx, d)
    psi = diag_step(psi, 0.5 * dt, c0, c1, q, d, V)
    psi = offdiag_step(psi, dt, c1, d)
    psi = diag_step(psi, 0.5 * dt, c0, c1, q, d, V)
    psi = kinetic(psi, 0.5 * dt, dx, d)
    return psi


# ----------------------------------------------------------------------------------
# Alternative local step: exact spin rotation (same Eq. (GPE), different splitting)
# ----------------------------------------------------------------------------------
#
# The interaction part of Eq. (GPE) equals c0 rho + c1 F.f + q f_z^2 applied to psi, with
# f the spin-1 matrices and F = psi^+ f psi the local spin.  The flow of c0 rho + c1 F.f
# keeps rho and F fixed, so over a time tau it is exactly
#   psi <- exp(-i c0 rho tau) exp(-i c1 tau F.f) psi,
# and for spin 1, (u.f)^3 = u.f for a unit vector u, giving
#   exp(-i th u.f) = 1 - i sin(th) u.f + (cos(th) - 1) (u.f)^2,  th = c1 tau |F|.
# The q f_z^2 phase is split symmetrically around it.

def spin_dot_f(F_z, F_p, p1, p0, pm):
    """(F.f) psi with F.f = [[F_z, F_-/sqrt2, 0], [F_+/sqrt2, 0, F_-/sqrt2], [0, F_+/sqrt2, -F_z]],
    F_+ = F_x + i F_y, F_- = conj(F_+)."""
    r2 = math.sqrt(2.0)
    F_m = F_p.conj()
    return F_z * p1 + F_m / r2 * p0, F_p / r2 * p1 + F_m / r2 * pm, F_p / r2 * p0 - F_z * pm


def rotation_interaction(psi, tau, c0, c1, d):
    """exp(-i c0 rho tau) exp(-i c1 tau F.f) psi per site (F, rho of the input)."""
    p1, p0, pm = psi.select(-d - 1, 0), psi.select(-d - 1, 1), psi.select(-d - 1, 2)
    n1, n0, nm = (p1.abs() ** 2), (p0.abs() ** 2), (pm.abs() ** 2)
    rho = n1 + n0 + nm
    F_z = n1 - nm
    F_p = transverse_spin(psi, d)
    Fabs2 = F_z ** 2 + F_p.real ** 2 + F_p.imag ** 2
    zero = Fabs2 == 0
    Fabs = torch.sqrt(torch.where(zero, torch.ones_like(Fabs2), Fabs2))
    th = c1 * tau * Fabs
    g1, g0, gm = spin_dot_f(F_z, F_p, p1, p0, pm)
    h1, h0, hm = spin_dot_f(F_z, F_p, g1, g0, gm)
    s = torch.where(zero, torch.zeros_like(th), torch.sin(th) / Fabs)
    c = torch.where(zero, torch.zeros_like(th), (torch.cos(th) - 1.0) / (Fabs * Fabs))
    ph = torch.exp(-1j * c0 * tau * rho)
    out = [ph * (p - 1j * s * g + c * h) for p, g, h in ((p1, g1, h1), (p0, g0, h0), (pm, gm, hm))]
    return torch.stack(out, dim=-d - 1)


def quadratic_zeeman(psi, tau, q, d, V=None):
    """exp(-i (q f_z^2 + V) tau): psi_+-1 pick up exp(-i q tau), psi_0 is unchanged by q;
    with a potential each psi_m also picks up exp(-i V_m tau)."""
    phase = torch.exp(torch.as_tensor(-1j * q * tau, dtype=CDT))
    out = torch.stack([psi.select(-d - 1, 0) * phase, psi.select(-d - 1, 1), psi.select(-d - 1, 2) * phase],
                      dim=-d - 1)
    if V is not None:
        out = out * torch.exp(-1j * tau * torch.as_tensor(V, dtype=RDT))
    return out


def strang_step_rotation(psi, dt, c0, c1, q, dx, d, V=None):
    """K(dt/2) Q(dt/2) R(dt) Q(dt/2) K(dt/2) with R the exact rotation above and Q the
    quadratic Zeeman phase (and the potential, which is diagonal too)."""
    psi = kinetic(psi, 0.5 * dt, dx, d)
    psi = quadratic_zeeman(psi, 0.5 * dt, q, d, V)
    psi = rotation_interaction(psi, dt, c0, c1, d)
    psi = quadratic_zeeman(psi, 0.5 * dt, q, d, V)
    psi = kinetic(psi, 0.5 * dt, dx, d)
    return psi


def propagate_rotation(psi, dt, nsteps, c0, c1, q, dx, d, t0=0.0, V=None):
    for n in range(nsteps):
        qn = q(t0 + (n + 0.5) * dt) if callable(q) else q
        psi = strang_step_rotation(psi, dt, c0, c1, qn, dx, d, V)
    return psi


def q_piecewise_linear(knots, t_end):
    """q(t): piecewise-linear through knots at t_j = j t_end / (K - 1), clamped outside.

    ``knots`` may be a tensor with requires_grad (gradients w.r.t. the knots).
    """
    knots = torch.as_tensor(knots, dtype=RDT)
    K = knots.shape[0]

    def q_of_t(t):
        if K == 1:
            return knots[0]
        u = t / t_end * (K - 1)
        if u <= 0.0:
            return knots[0]
        if u >= K - 1:
            return knots[K - 1]
        i = int(math.floor(u))
        w = u - i
        return knots[i] * (1.0 - w) + knots[i + 1] * w

    return q_of_t


def propagate(psi, dt, nsteps, c0, c1, q, dx, d, t0=0.0, V=None):
    """nsteps Strang steps from time t0.  q: number or callable q(t) evaluated at the
    step midpoint t0 + (n + 1/2) dt.  V: optional potential (3, *shape)."""
    for n in range(nsteps):
        qn = q(t0 + (n + 0.5) * dt) if callable(q) else q
        psi = strang_step(psi, dt, c0, c1, qn, dx, d, V)
    return psi


# ----------------------------------------------------------------------------------
# Observables (Sec. 2.1; normalisations: reading R7)
# ----------------------------------------------------------------------------------

def transverse_spin(psi, d):
    """F_perp = F_x + i F_y = sqrt(2) (psi_1^* psi_0 + psi_0^* psi_-1)."""
    p1, p0, pm = psi.select(-d - 1, 0), psi.select(-d - 1, 1), psi.select(-d - 1, 2)
    return math.sqrt(2.0) * (p1.conj() * p0 + p0.conj() * pm)


def occupation_modes(psi, dx, d):
    """n_m(k) = |A_m(k)|^2 - 1/2 per grid mode, A_m(k) = dx^d / sqrt(L^d) sum_x psi_m e^{-ikx}."""
    shape = _spatial_shape(psi, d)
    ntot = math.prod(shape)
    A = torch.fft.fftn(psi, dim=_dims(d)) * (dx ** d / math.sqrt(ntot * dx ** d))
    return A.real ** 2 + A.imag ** 2 - 0.5


def spin_structure_modes(psi, dx, d):
    """S_perp(k) = |F_perp(k)|^2 / L^d per grid mode, F_perp(k) = dx^d sum_x F_perp e^{-ikx}
    (Sec. 2.1, structure factor before the ensemble average)."""
    shape = _spatial_shape(psi, d)
    ntot = math.prod(shape)
    F = torch.fft.fftn(transverse_spin(psi, d), dim=_dims(d)) * dx ** d
    return (F.real ** 2 + F.imag ** 2) / (ntot * dx ** d)


def radial_bins(shape):
    """Radial bin of every mode: b = round(|j|) with j the folded integer mode vector
    (|k| / (2 pi / L) for equal side lengths L).  sqrt(m) is never a half integer for
    integer m, so the rounding has no ties."""
    if len(set(shape)) != 1:
        raise ValueError("radial binning needs equal side lengths")
    d = len(shape)
    m = torch.zeros(shape, dtype=torch.int64)
    for ax, n in enumerate(shape):
        j = torch.fft.fftfreq(n, d=1.0 / n, dtype=RDT).round().to(torch.int64)
        view = [1] * d
        view[ax] = n
        m = m + (j * j).reshape(view)
    b = torch.round(torch.sqrt(m.to(RDT))).to(torch.int64)
    return b


def bin_sum(values, bins):
    """Sum of ``values[..., modes]`` into radial bins (last d axes are modes)."""
    nb = int(bins.max()) + 1
    flat = values.reshape(values.shape[:values.dim() - bins.dim()] + (-1,))
    out = torch.zeros(flat.shape[:-1] + (nb,), dtype=flat.dtype)
    return out.index_add_(-1, bins.reshape(-1), flat)


def bin_counts(shape):
    b = radial_bins(shape).reshape(-1)
    return torch.bincount(b)


def diagnostics(psi, dx, c0, c1, q, d, V=None):
    """N_m, and the energy split into kinetic, q, c0, c1 and potential parts (FP64).

    E = dx^d sum_x [ sum_m psi_m^* (-Laplacian/2) psi_m + q (n_1 + n_-1)
                     + c0/2 rho^2 + c1/2 (F_z^2 + |F_perp|^2) + sum_m V_m n_m ],
    whose functional derivative d E / d psi_m^* reproduces the bracket of Eq. (GPE);
    the Laplacian is the spectral one (Parseval over the grid modes).
    Returns a tensor (..., 8): N_1, N_0, N_-1, E_kin, E_q, E_c0, E_c1, E_V (E_V = 0
    without a potential).
    """
    shape = _spatial_shape(psi, d)
    ntot = math.prod(shape)
    vol = dx ** d
    n = psi.real ** 2 + psi.imag ** 2
    sp = _dims(d)
    N = n.sum(dim=sp) * vol
    pk = torch.fft.fftn(psi, dim=sp)
    ekin = (0.5 * k_squared(shape, dx) * (pk.real ** 2 + pk.imag ** 2)).sum(dim=sp).sum(-1) * vol / ntot
    n1, n0, nm = n.select(-d - 1, 0), n.select(-d - 1, 1), n.select(-d - 1, 2)
    rho = n1 + n0 + nm
    fz = n1 - nm
    fp = transverse_spin(psi, d)
    eq = q * (n1 + nm).sum(dim=sp) * vol
    ec0 = 0.5 * c0 * (rho * rho).sum(dim=sp) * vol
    ec1 = 0.5 * c1 * (fz * fz + fp.real ** 2 + fp.imag ** 2).sum(dim=sp) * vol
    if V is None:
        ev = torch.zeros_like(ec1)
    else:
        ev = (torch.as_tensor(V, dtype=RDT) * n).sum(dim=sp).sum(-1) * vol
    return torch.cat([N, torch.stack([ekin, eq, ec0, ec1, ev], dim=-1)], dim=-1)


def larmor_angle(psi, d):
    """phi_L = arg(F_x + i F_y), the orientation of the transverse spin (Sec. 1, Fig. 1)."""
    return torch.angle(transverse_spin(psi, d))


def winding_number(psi):
    """Q_w / (2 pi) of a 1D periodic trajectory (Sec. 1, Fig. 1: Q_w = int dx d_x phi_L):
    the sum over neighbouring sites of the Larmor-angle increment arg(F(x)^* F(x+1)),
    each in (-pi, pi], around the ring, divided by 2 pi.  An integer up to rounding
    whenever F_perp has no zeros.  psi: (..., 3, n)."""
    F = transverse_spin(psi, 1)
    inc = torch.angle(F.conj() * torch.roll(F, -1, dims=-1))
    return inc.sum(dim=-1) / (2.0 * math.pi)


def sf_band_loss(psi, dx, d, kmin, kmax):
    """Late-time loss: mean over trajectories of sum_{k: kmin <= |k| <= kmax} S_perp(k),
    summed over grid modes, bounds inclusive.  psi: (ntraj, 3, *shape)."""
    shape = _spatial_shape(psi, d)
    kabs = torch.sqrt(k_squared(shape, dx))
    mask = (kabs >= kmin) & (kabs <= kmax)
    S = spin_structure_modes(psi, dx, d)
    return (S * mask).sum(dim=_dims(d)).mean()
