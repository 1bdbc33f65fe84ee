"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Every pin here comes from something other than the oracle itself: published test
vectors, closed-form solutions of Eq. (GPE) in special cases, a library matrix
exponential, an independent ODE integrator, brute-force sums on tiny grids,
conservation laws, the scheme's convergence order and statistics of the noise.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import torch

from oracle import gpe_oracle as O
from oracle.philox import philox4x32_10, tw_noise
from paper_2310_03636_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def T(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128)


# ---------------------------------------------------------------- random numbers

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(tuple(v[0:4]), tuple(v[4:6]))
        assert [int(o) for o in out] == v[6:10]


def test_noise_statistics():
    """<|eta|^2> = noise_per_mode / dx^d, complex Gaussian (<|eta|^4> = 2 <|eta|^2>^2),
    zero mean, independent components, seed/trajectory dependence."""
    shape, dx, npm = (64, 64), 0.5, 0.5
    eta = tw_noise(shape, seed=123, traj=3, noise_per_mode=npm, dx=dx)
    s2 = npm / dx ** 2
    p = np.abs(eta) ** 2
    nsamp = p.size
    assert abs(p.mean() - s2) < 4 * s2 / math.sqrt(nsamp)
    assert abs((p ** 2).mean() / s2 ** 2 - 2.0) < 0.1
    assert abs(eta.mean()) < 4 * math.sqrt(s2 / nsamp)
    c = np.mean(eta[0] * eta[1].conj()) / s2
    assert abs(c) < 4 / math.sqrt(eta[0].size)
    assert np.array_equal(eta, tw_noise(shape, 123, 3, npm, dx))
    assert not np.allclose(eta, tw_noise(shape, 123, 4, npm, dx))
    assert not np.allclose(eta, tw_noise(shape, 124, 3, npm, dx))


# ---------------------------------------------------------------- kinetic step

@pytest.mark.parametrize("shape,js,dx", [
    ((32,), [(5,), (-3,), (16,)], 0.7),
    ((16, 32), [(3, -5), (-8, 1), (0, 7)], 0.7),
    ((8, 4, 16), [(1, -2, 3), (4, 1, -8), (-3, 0, 5)], 1.3),
])
def test_kinetic_plane_wave(shape, js, dx):
    """A plane wave e^{ik.x} only picks up the phase e^{-i tau |k|^2 / 2}.
    Different wave vectors per component and axis catch a transposed axis or a wrong k."""
    d = len(shape)
    psi = np.stack([W.plane_wave(shape, j, dx) for j in js])
    tau = 0.37
    out = O.kinetic(T(psi), tau, dx, d).numpy()
    for m, j in enumerate(js):
        k2 = sum((2 * np.pi * ji / (n * dx)) ** 2 for n, ji in zip(shape, j))
        np.testing.assert_allclose(out[m], psi[m] * np.exp(-0.5j * tau * k2), atol=1e-12)


def test_free_gaussian_spreading():
    """c0 = c1 = q = 0: a Gaussian exp(-x^2 / (2 s0)) evolves as
    (s0 / s)^{1/2} exp(-x^2 / (2 s)), s = s0 + i t (free Schroedinger, hbar = m = 1)."""
    n, dx, sig = 1024, 0.1, 1.0
    x = (np.arange(n) - n // 2) * dx
    psi = np.zeros((3, n), complex)
    psi[1] = np.exp(-x ** 2 / (2 * sig ** 2))
    dt, steps = 0.05, 40
    out = O.propagate(T(psi), dt, steps, 0.0, 0.0, 0.0, dx, 1).numpy()
    t = dt * steps
    s = sig ** 2 + 1j * t
    exact = np.sqrt(sig ** 2 / s) * np.exp(-x ** 2 / (2 * s))
    np.testing.assert_allclose(out[1], exact, atol=1e-12)
    assert np.abs(out[0]).max() == 0 and np.abs(out[2]).max() == 0


def test_free_gaussian_2d_width():
    """2D isotropic Gaussian in m = +1: |psi|^2 width grows as sqrt(s0^2 + t^2)/s0."""
    n, dx, sig = 128, 0.25, 1.2
    x = (np.arange(n) - n // 2) * dx
    r2 = x[:, None] ** 2 + x[None, :] ** 2
    psi = np.zeros((3, n, n), complex)
    psi[0] = np.exp(-r2 / (2 * sig ** 2))
    t = 1.5
    out = O.propagate(T(psi), 0.1, 15, 0.0, 0.0, 0.0, dx, 2).numpy()
    s = sig ** 2 + 1j * t
    exact = (sig ** 2 / s) * np.exp(-r2 / (2 * s))
    np.testing.assert_allclose(out[0], exact, atol=1e-12)


# ---------------------------------------------------------------- diagonal step

@pytest.mark.parametrize("c1", [-0.1, 0.25])
def test_uniform_polar_phase(c1):
    """psi_0 = sqrt(n), psi_+-1 = 0 is stationary up to exp(-i c0 n t) (mu = c0 n)."""
    n, c0, q, dt, steps = 1.3, 1.0, 0.09, 0.01, 50
    psi = np.zeros((3, 16, 16), complex)
    psi[1] = math.sqrt(n)
    out = O.propagate(T(psi), dt, steps, c0, c1, q, 1.0, 2).numpy()
    t = dt * steps
    np.testing.assert_allclose(out[1], math.sqrt(n) * np.exp(-1j * c0 * n * t), atol=1e-13)
    assert np.abs(out[0]).max() == 0 and np.abs(out[2]).max() == 0


@pytest.mark.parametrize("comp", [0, 2])
def test_uniform_ferro_phase(comp):
    """psi_{+-1} = sqrt(n) alone: phase exp(-i (q + (c0 + c1) n) t)."""
    n, c0, c1, q, dt, steps = 0.8, 1.0, -0.1, 0.09, 0.02, 30
    psi = np.zeros((3, 32), complex)
    psi[comp] = math.sqrt(n)
    out = O.propagate(T(psi), dt, steps, c0, c1, q, 1.0, 1).numpy()
    t = dt * steps
    np.testing.assert_allclose(out[comp], math.sqrt(n) * np.exp(-1j * (q + (c0 + c1) * n) * t),
                               atol=1e-13)


def test_uniform_two_component_phases():
    """psi_1 = sqrt(n1), psi_-1 = sqrt(nm), psi_0 = 0: a = b = 0 so only the diagonal acts;
    f_1 = q + (c0+c1) rho - 2 c1 nm and f_-1 = q + (c0+c1) rho - 2 c1 n1 differ."""
    n1, nm, c0, c1, q, dt, steps = 0.7, 0.2, 1.0, -0.1, 0.05, 0.02, 25
    psi = np.zeros((3, 8, 8), complex)
    psi[0] = math.sqrt(n1)
    psi[2] = math.sqrt(nm)
    out = O.propagate(T(psi), dt, steps, c0, c1, q, 1.0, 2).numpy()
    t, rho = dt * steps, n1 + nm
    np.testing.assert_allclose(out[0], math.sqrt(n1) * np.exp(-1j * (q + (c0 + c1) * rho - 2 * c1 * nm) * t),
                               atol=1e-13)
    np.testing.assert_allclose(out[2], math.sqrt(nm) * np.exp(-1j * (q + (c0 + c1) * rho - 2 * c1 * n1) * t),
                               atol=1e-13)


# ---------------------------------------------------------------- off-diagonal step

def test_offdiag_matrix_is_expm():
    """The printed 3x3 matrix (reading: ab(cos - 1)) equals expm(-i c1 dt S) for
    S = [[0, a, 0], [a*, 0, b], [0, b*, 0]], computed by scipy (Pade), and is unitary."""
    g = np.random.default_rng(7)
    for _ in range(20):
        a, b = g.normal(size=2) + 1j * g.normal(size=2)
        c1dt = g.normal() * 0.8
        S = np.array([[0, a, 0], [np.conj(a), 0, b], [0, np.conj(b), 0]])
        Uref = scipy.linalg.expm(-1j * c1dt * S)
        lam2 = torch.tensor(abs(a) ** 2 + abs(b) ** 2, dtype=torch.float64)
        U = O.offdiag_matrix(T(a), T(b), c1dt, lam2)
        Um = np.array([[complex(U[i][j]) for j in range(3)] for i in range(3)])
        np.testing.assert_allclose(Um, Uref, atol=1e-13)
        np.testing.assert_allclose(Um.conj().T @ Um, np.eye(3), atol=1e-13)
    U0 = O.offdiag_matrix(T(0j), T(0j), 0.3, torch.tensor(0.0, dtype=torch.float64))
    assert np.allclose([[complex(U0[i][j]) for j in range(3)] for i in range(3)], np.eye(3))


def _rk4_offdiag_flow(psi, c1, tau, nsub=2000):
    """Independent reference: RK4 of the pure spin-mixing flow i psi' = c1 S(psi) psi."""
    def rhs(p):
        p1, p0, pm = p
        a, b = np.conj(pm) * p0, np.conj(p0) * p1
        return -1j * c1 * np.array([a * p0, np.conj(a) * p1 + b * pm, np.conj(b) * p0])
    h = tau / nsub
    p = np.array(psi, complex)
    for _ in range(nsub):
        k1 = rhs(p)
        k2 = rhs(p + 0.5 * h * k1)
        k3 = rhs(p + 0.5 * h * k2)
        k4 = rhs(p + h * k3)
        p = p + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return p


def test_offdiag_step_local_order_three():
    """The predictor-averaged matrix step has local error O(tau^3) against the exact
    spin-mixing flow: halving tau divides the error by ~8."""
    g = np.random.default_rng(11)
    psi = g.normal(size=3) + 1j * g.normal(size=3)
    c1 = -0.9
    errs = []
    for tau in (0.05, 0.025, 0.0125):
        ref = _rk4_offdiag_flow(psi, c1, tau, nsub=400)
        out = O.offdiag_step(T(psi.reshape(3, 1)), tau, c1, 1).numpy().ravel()
        errs.append(np.linalg.norm(out - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.0 and 7.0 < r2 < 9.0, errs
    # the step is unitary: norm of the spinor conserved
    out = O.offdiag_step(T(psi.reshape(3, 1)), 0.3, c1, 1).numpy().ravel()
    assert abs(np.linalg.norm(out) - np.linalg.norm(psi)) < 1e-13


# ---------------------------------------------------------------- the scheme

def _bogoliubov_modes(A, B, t):
    """Linear pair i u' = A u + B v, i v' = -B u - A v with u(0) = 1, v(0) = 0."""
    E2 = complex(A * A - B * B)
    E = np.sqrt(E2)
    if abs(E) < 1e-14:
        c, s = 1.0, t
    else:
        c, s = np.cos(E * t), np.sin(E * t) / E
    return c - 1j * A * s, 1j * B * s


@pytest.mark.parametrize("q,j", [(0.09, 2), (0.09, 9), (0.35, 3)])
def test_bogoliubov_spin_modes(q, j):
    """Linearising Eq. (GPE) around the polar state psi_0 = sqrt(n) e^{-i c0 n t} gives,
    for u = psi_1(k) and v = conj(psi_-1(-k)) (rotating frame), A = eps_k + q + c1 n,
    B = c1 n, E_s = sqrt((eps_k + q)(eps_k + q + 2 c1 n)); unstable band included."""
    N, dx, n, c0, c1 = 64, 1.0, 1.0, 1.0, -0.1
    eps0 = 1e-7
    x = np.arange(N) * dx
    k = 2 * np.pi * j / (N * dx)
    psi = np.zeros((3, N), complex)
    psi[1] = math.sqrt(n)
    psi[0] = eps0 * np.exp(1j * k * x)
    dt, steps = 0.01, 1500
    out = O.propagate(T(psi), dt, steps, c0, c1, q, dx, 1).numpy()
    t = dt * steps
    rot = np.exp(1j * c0 * n * t)
    u = np.fft.fft(out[0] * rot)[j] / N / eps0
    v = np.conj(np.fft.fft(out[2] * rot)[(-j) % N] / N) / eps0
    A, B = 0.5 * k * k + q + c1 * n, c1 * n
    ue, ve = _bogoliubov_modes(A, B, t)
    assert abs(u - ue) < 2e-3 * max(1.0, abs(ue))
    assert abs(v - ve) < 2e-3 * max(1.0, abs(ue))


@pytest.mark.parametrize("j", [1, 6])
def test_bogoliubov_density_mode(j):
    """Density (phonon) branch around the polar state: A = eps_k + c0 n, B = c0 n,
    E_d = sqrt(eps_k (eps_k + 2 c0 n))."""
    N, dx, n, c0, c1, q = 32, 0.8, 1.5, 1.0, -0.1, 0.09
    eps0 = 1e-7
    x = np.arange(N) * dx
    k = 2 * np.pi * j / (N * dx)
    psi = np.zeros((3, N), complex)
    psi[1] = math.sqrt(n) + eps0 * np.exp(1j * k * x)
    dt, steps = 0.005, 1000
    out = O.propagate(T(psi), dt, steps, c0, c1, q, dx, 1).numpy()
    t = dt * steps
    f = np.fft.fft(out[1] * np.exp(1j * c0 * n * t)) / N / eps0
    A, B = 0.5 * k * k + c0 * n, c0 * n
    ue, ve = _bogoliubov_modes(A, B, t)
    assert abs(f[j] - ue) < 2e-3 * max(1.0, abs(ue))
    assert abs(np.conj(f[(-j) % N]) - ve) < 2e-3 * max(1.0, abs(ue))


def test_norm_conservation():
    """Every sub-step is unitary: the total norm is conserved to rounding."""
    psi = T(W.random_field((32, 32), 2, seed=5, scale=0.7))
    out = O.propagate(psi, 0.02, 40, 1.0, -0.1, 0.09, 1.0, 2)
    n0 = (psi.abs() ** 2).sum(dim=(1, 2, 3))
    n1 = (out.abs() ** 2).sum(dim=(1, 2, 3))
    assert torch.allclose(n0, n1, rtol=1e-12, atol=0)


def test_second_order_convergence():
    """Global error against a fine-step run scales as dt^2 (Strang splitting)."""
    psi = T(W.smooth_random_field((64,), 1, seed=9))
    Tend = 1.0
    ref = O.propagate(psi, Tend / 512, 512, 1.0, -0.5, 0.09, 1.0, 1)
    errs = []
    for nst in (10, 20, 40):
        out = O.propagate(psi, Tend / nst, nst, 1.0, -0.5, 0.09, 1.0, 1)
        errs.append(float((out - ref).abs().pow(2).sum().sqrt()))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_energy_and_fz_drift_second_order():
    """Energy and F_z are conserved by Eq. (GPE); the scheme drifts by O(dt^2)."""
    psi = T(W.smooth_random_field((64,), 1, seed=3))
    c0, c1, q, dx = 1.0, -0.5, 0.09, 1.0

    def en_fz(p):
        dg = O.diagnostics(p, dx, c0, c1, q, 1)[0]
        return float(dg[3:].sum()), float(dg[0] - dg[2])
    E0, F0 = en_fz(psi)
    dE, dF = [], []
    for nst in (10, 20, 40):
        out = O.propagate(psi, 2.0 / nst, nst, c0, c1, q, dx, 1)
        E1, F1 = en_fz(out)
        dE.append(abs(E1 - E0))
        dF.append(abs(F1 - F0))
    assert 3.0 < dE[0] / dE[1] < 5.0 and 3.0 < dE[1] / dE[2] < 5.0, dE
    assert 3.0 < dF[0] / dF[1] < 5.0 and 3.0 < dF[1] / dF[2] < 5.0, dF


def test_energy_functional_generates_gpe():
    """dE/d psi^* equals the operator of Eq. (GPE) applied to psi (written here from the
    equation itself), so the energy diagnostic is the conserved quantity of the flow."""
    shape, dx, c0, c1, q = (12, 10), 0.9, 1.1, -0.3, 0.2
    psi = T(W.random_field(shape, 1, seed=21, scale=0.5)[0]).requires_grad_(True)
    E = O.diagnostics(psi, dx, c0, c1, q, 2)[3:].sum()
    (g,) = torch.autograd.grad(E, psi)
    lhs = 0.5 * g / dx ** 2                       # torch grad = 2 dE/dpsi^*; per-site volume dx^d
    p = psi.detach().numpy()
    p1, p0, pm = p
    n1, n0, nm = abs(p1) ** 2, abs(p0) ** 2, abs(pm) ** 2
    rho = n1 + n0 + nm
    ky = 2 * np.pi * np.fft.fftfreq(shape[0], dx)
    kx = 2 * np.pi * np.fft.fftfreq(shape[1], dx)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    lap = lambda f: np.fft.ifft2(-k2 * np.fft.fft2(f))
    M = [[-2 * nm, np.conj(pm) * p0, 0 * p0],
         [pm * np.conj(p0), -n0 - q / c1, np.conj(p0) * p1],
         [0 * p0, p0 * np.conj(p1), -2 * n1]]
    H = []
    for i in range(3):
        h = -0.5 * lap(p[i]) + (q + (c0 + c1) * rho) * p[i]
        h = h + c1 * sum(M[i][j] * p[j] for j in range(3))
        H.append(h)
    np.testing.assert_allclose(lhs.numpy(), np.array(H), atol=1e-12)


# ---------------------------------------------------------------- external potential

@pytest.mark.parametrize("rotation", [False, True])
def test_potential_linear_zeeman_and_uniform_shift(rotation):
    """V_m = v + p m is a global phase plus a linear Zeeman term; both commute with
    every part of Eq. (GPE) (the interaction depends on psi only through rho, F_z and
    F_perp's modulus, and the mixing terms conserve F_z), and the split step is covariant
    under psi_m -> exp(-i p m t) psi_m, so psi_m(t) = exp(-i (v + p m) t) psi_m^{V=0}(t)."""
    shape, dx, c0, c1, q, dt, n = (32, 16), 1.0, 1.0, -0.4, 0.07, 0.05, 12
    psi = T(W.smooth_random_field(shape, 1, seed=17))
    v, pz = 0.3, -0.45
    V = np.stack([np.full(shape, v + pz), np.full(shape, v), np.full(shape, v - pz)])
    prop = O.propagate_rotation if rotation else O.propagate
    ref = prop(psi, dt, n, c0, c1, q, dx, 2)
    out = prop(psi, dt, n, c0, c1, q, dx, 2, V=V)
    ph = np.exp(-1j * (v + pz * np.array([1.0, 0.0, -1.0])) * n * dt).reshape(1, 3, 1, 1)
    np.testing.assert_allclose(out.numpy(), ref.numpy() * ph, atol=1e-12)


def test_potential_linear_limit_converges_to_exact_propagator():
    """c0 = c1 = q = 0: Eq. (GPE) is the linear Schroedinger equation
    i d psi_m / dt = (-Laplacian/2 + V_m) psi_m.  On the periodic grid its exact solution is
    expm(-i H_m t) psi_m with H_m the dense grid Hamiltonian (spectral Laplacian); the
    split step must converge to it at second order in dt (a wrong sign or a missing half
    of V in D would leave an O(1) error)."""
    n, dx, t_end = 48, 0.7, 1.2
    V = W.smooth_potential((n,), seed=5, amp=0.8, dx=dx)
    psi = T(W.smooth_random_field((n,), 1, seed=9))
    k = 2 * np.pi * np.fft.fftfreq(n, dx)
    F = np.fft.fft(np.eye(n), axis=0)
    lap_k = F.conj().T @ np.diag(0.5 * k * k) @ F / n            # -Laplacian/2 on the grid
    exact = np.stack([scipy.linalg.expm(-1j * t_end * (lap_k + np.diag(V[m]))) @ psi.numpy()[0, m]
                      for m in range(3)])
    errs = []
    for nst in (12, 24, 48):
        out = O.propagate(psi, t_end / nst, nst, 0.0, 0.0, 0.0, dx, 1, V=V).numpy()[0]
        errs.append(np.sqrt((abs(out - exact) ** 2).sum() / (abs(exact) ** 2).sum()))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
    assert errs[-1] < 1e-3


def test_potential_energy_conserved_second_order():
    """With a potential the conserved energy includes E_V = dx^d sum V_m n_m; the split step
    conserves the total to O(dt^2), while E_V alone changes by far more (the cloud moves
    in the well), so a dropped or mis-signed E_V breaks the pin."""
    n, dx, c0, c1, q = 64, 1.0, 1.0, -0.5, 0.09
    V = W.smooth_potential((n,), seed=12, amp=0.05)
    psi = T(W.smooth_random_field((n,), 1, seed=3))
    dg0 = O.diagnostics(psi, dx, c0, c1, q, 1, V=V)[0]
    dE, dEV = [], []
    for nst in (10, 20, 40):
        dg1 = O.diagnostics(O.propagate(psi, 2.0 / nst, nst, c0, c1, q, dx, 1, V=V), dx, c0, c1, q, 1, V=V)[0]
        dE.append(abs(float(dg1[3:].sum() - dg0[3:].sum())))
        dEV.append(abs(float(dg1[7] - dg0[7])))
    assert 3.0 < dE[0] / dE[1] < 5.0 and 3.0 < dE[1] / dE[2] < 5.0, dE
    assert dEV[-1] > 20 * dE[-1], (dEV, dE)


def test_potential_energy_functional_generates_gpe():
    """With V: dE/d psi_m^* gains V_m psi_m, the potential term of the bracket in the
    diagonal step of Sec. 2.2."""
    shape, dx, c0, c1, q = (12, 10), 0.9, 1.1, -0.3, 0.2
    V = W.smooth_potential(shape, seed=4, amp=0.7, dx=dx)
    psi = T(W.random_field(shape, 1, seed=21, scale=0.5)[0]).requires_grad_(True)
    (g0,) = torch.autograd.grad(O.diagnostics(psi, dx, c0, c1, q, 2)[3:].sum(), psi)
    (g1,) = torch.autograd.grad(O.diagnostics(psi, dx, c0, c1, q, 2, V=V)[3:].sum(), psi)
    diff = 0.5 * (g1 - g0) / dx ** 2
    np.testing.assert_allclose(diff.numpy(), V * psi.detach().numpy(), atol=1e-12)


def test_rotation_scheme_with_potential_keeps_fz():
    """A potential is diagonal in m, so the rotation scheme still conserves F_z to rounding."""
    shape, dx = (64,), 1.0
    V = W.smooth_potential(shape, seed=8, amp=0.3)
    psi = T(W.smooth_random_field(shape, 1, seed=3))
    out = O.propagate_rotation(psi, 0.05, 40, 1.0, -0.5, 0.09, dx, 1, V=V)
    d0 = O.diagnostics(psi, dx, 1.0, -0.5, 0.09, 1)[0]
    d1 = O.diagnostics(out, dx, 1.0, -0.5, 0.09, 1)[0]
    assert abs(float((d1[0] - d1[2]) - (d0[0] - d0[2]))) < 1e-12
    assert float((out - O.propagate_rotation(psi, 0.05, 40, 1.0, -0.5, 0.09, dx, 1)).abs().max()) > 1e-3


# ---------------------------------------------------------------- Larmor angle, winding

@pytest.mark.parametrize("j1,j0,jm", [(0, 3, 0), (2, 0, 0), (0, 0, -5), (1, -2, 0), (0, 0, 0)])
def test_winding_number_of_phase_windings(j1, j0, jm):
    """psi_1 = a e^{2 pi i j1 x/L}, psi_0 = b e^{2 pi i j0 x/L}, psi_-1 = 0: F_perp is
    proportional to e^{2 pi i (j0 - j1) x/L}, so Q_w / 2 pi = j0 - j1; with psi_1 = 0 and
    psi_-1 = c e^{2 pi i jm x/L} instead, F_perp ~ e^{2 pi i (jm - j0) x/L}."""
    n = 128
    x = np.arange(n)
    a, b, c = 0.6, 0.9 * np.exp(0.4j), 0.7
    if jm == 0:
        psi = np.stack([a * np.exp(2j * np.pi * j1 * x / n), b * np.exp(2j * np.pi * j0 * x / n), 0 * x])
        want = j0 - j1
    else:
        psi = np.stack([0 * x, b * np.exp(2j * np.pi * j0 * x / n), c * np.exp(2j * np.pi * jm * x / n)])
        want = jm - j0
    assert abs(float(O.winding_number(T(psi))) - want) < 1e-12
    phi = O.larmor_angle(T(psi), 1).numpy()
    np.testing.assert_allclose(np.exp(1j * phi), np.exp(1j * (np.angle(np.conj(psi[0]) * psi[1] + np.conj(psi[1]) * psi[2]))),
                               atol=1e-12)


def test_winding_number_against_unwrap_and_symmetries():
    """Random spinors: an integer equal to the net turn of numpy's unwrapped Larmor angle,
    unchanged by a global phase and by a spin rotation about z (F_perp -> e^{-i a} F_perp)."""
    n = 256
    for seed in range(6):
        psi = W.random_field((n,), 1, seed=100 + seed, scale=0.8, mean=(0.3, 0.2, 0.1))[0]
        w = float(O.winding_number(T(psi)))
        assert abs(w - round(w)) < 1e-10
        F = math.sqrt(2.0) * (np.conj(psi[0]) * psi[1] + np.conj(psi[1]) * psi[2])
        ang = np.unwrap(np.angle(np.append(F, F[0])))
        assert abs((ang[-1] - ang[0]) / (2 * np.pi) - w) < 1e-10
        rot = psi * np.exp(-1j * 0.7 * np.array([1.0, 0.0, -1.0]))[:, None] * np.exp(0.3j)
        assert abs(float(O.winding_number(T(rot))) - w) < 1e-10


# ---------------------------------------------------------------- observables

def _brute_dft(f, dx):
    """sum_x f(x) e^{-i k.x} by explicit loops (tiny grids only)."""
    shape = f.shape
    d = len(shape)
    out = np.zeros(shape, complex)
    idx = list(np.ndindex(*shape))
    for kk in idx:
        s = 0j
        for xx in idx:
            ph = sum(2 * np.pi * kk[a] * xx[a] / shape[a] for a in range(d))
            s += f[xx] * np.exp(-1j * ph)
        out[kk] = s
    return out


def test_spectra_brute_force():
    shape, dx = (6, 4), 0.5
    d = 2
    psi = W.random_field(shape, 1, seed=33, scale=0.8)[0]
    L = shape[0] * dx
    vol = dx ** d
    ntot = math.prod(shape)
    nm = O.occupation_modes(T(psi), dx, d).numpy()
    for m in range(3):
        A = vol / math.sqrt(ntot * vol) * _brute_dft(psi[m], dx)
        np.testing.assert_allclose(nm[m], abs(A) ** 2 - 0.5, atol=1e-12)
    Fp = math.sqrt(2) * (np.conj(psi[0]) * psi[1] + np.conj(psi[1]) * psi[2])
    S = abs(vol * _brute_dft(Fp, dx)) ** 2 / (ntot * vol)
    np.testing.assert_allclose(O.spin_structure_modes(T(psi), dx, d).numpy(), S, atol=1e-12)


def test_parseval_occupation():
    """sum_k |A_m(k)|^2 = N_m = dx^d sum_x |psi_m|^2."""
    shape, dx = (16, 16, 8), 0.7
    psi = T(W.random_field(shape, 1, seed=4)[0])
    nk = O.occupation_modes(psi, dx, 3) + 0.5
    N = O.diagnostics(psi, dx, 1.0, -0.1, 0.0, 3)[:3]
    assert torch.allclose(nk.sum(dim=(1, 2, 3)), N, rtol=1e-12)


def test_kinetic_energy_brute_force():
    shape, dx = (5, 6), 0.8
    psi = W.random_field(shape, 1, seed=8)[0]
    ekin = 0.0
    for m in range(3):
        f = _brute_dft(psi[m], dx)
        for kk in np.ndindex(*shape):
            k2 = sum((2 * np.pi * (kk[a] if kk[a] <= shape[a] // 2 else kk[a] - shape[a]) / (shape[a] * dx)) ** 2
                     for a in range(2))
            ekin += 0.5 * k2 * abs(f[kk]) ** 2
    ekin *= dx ** 2 / math.prod(shape)
    dg = O.diagnostics(T(psi), dx, 1.0, -0.1, 0.0, 2)
    assert abs(float(dg[3]) - ekin) < 1e-12 * max(1.0, ekin)


@pytest.mark.parametrize("shape", [(256,), (16, 16), (8, 8, 8), (512, 512)])
def test_radial_bins(shape):
    """b = round(|k| / dk) computed from floating-point |k| agrees with the integer rule;
    bin counts for 1D 256 and 2D 512^2 (129 and 363 bins)."""
    b = O.radial_bins(shape).numpy()
    if math.prod(shape) <= 4096:
        n = shape[0]
        L = n * 1.0
        for idx in np.ndindex(*shape):
            kk = [2 * np.pi * (i if i < n // 2 else i - n) / L for i in idx]
            assert b[idx] == int(np.floor(math.sqrt(sum(x * x for x in kk)) / (2 * np.pi / L) + 0.5))
    if shape == (256,):
        assert b.max() + 1 == 129
    if shape == (512, 512):
        assert b.max() + 1 == 363
        assert O.bin_counts(shape).sum() == 512 * 512


def test_bin_sum_explicit_loop():
    """Radial bin sums against an explicit loop over modes and leading indices, with values
    that differ per mode and per leading index (1D, 2D and 3D grids)."""
    g = np.random.default_rng(91)
    for lead, shape in (((3,), (16,)), ((2, 3), (8, 8)), ((2,), (4, 4, 4))):
        vals = g.normal(size=lead + shape)
        bins = O.radial_bins(shape).numpy()
        nb = int(bins.max()) + 1
        want = np.zeros(lead + (nb,))
        for li in np.ndindex(*lead):
            for mi in np.ndindex(*shape):
                want[li + (bins[mi],)] += vals[li + mi]
        got = O.bin_sum(torch.as_tensor(vals), torch.as_tensor(bins)).numpy()
        assert got.shape == want.shape
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
        # every mode lands in exactly one bin
        np.testing.assert_allclose(got.sum(-1), vals.reshape(lead + (-1,)).sum(-1), rtol=1e-12)


def test_sf_band_loss_brute_force():
    """Band loss = mean over trajectories of sum over grid modes with kmin <= |k| <= kmax of
    S_perp(k), from explicit DFT loops and an integer band rule.  On an 8 x 8 grid with
    dx = 1/2, |k| = (2 pi / 4) |j| for integer mode vectors j; kmin and kmax are put exactly
    on |j| = 1 and |j| = 2, so inclusive bounds take 12 modes and exclusive ones 4."""
    shape, dx, d = (8, 8), 0.5, 2
    psi = W.random_field(shape, 2, seed=58, scale=0.7)
    psi[1] *= 1.7     # trajectories differ in size: a sum instead of a mean is off by far more than 2x
    L = shape[0] * dx
    dk = 2 * math.pi / L
    jf = lambda i, n: i if i < n // 2 else i - n
    S = []
    for t in range(2):
        p = psi[t]
        Fp = math.sqrt(2) * (np.conj(p[0]) * p[1] + np.conj(p[1]) * p[2])
        S.append(abs(dx ** d * _brute_dft(Fp, dx)) ** 2 / L ** d)
    for (lo, hi), (mlo, mhi, incl) in (((dk, 2 * dk), (1, 4, True)),
                                       ((np.nextafter(dk, 9.0), np.nextafter(2 * dk, 0.0)), (1, 4, False))):
        want = 0.0
        count = 0
        for t in range(2):
            for kk in np.ndindex(*shape):
                m = sum(jf(kk[a], shape[a]) ** 2 for a in range(d))
                inside = (mlo <= m <= mhi) if incl else (mlo < m < mhi)
                if inside:
                    want += S[t][kk] / 2
                    count += 1
        assert count == 2 * (12 if incl else 4)
        got = float(O.sf_band_loss(T(psi), dx, d, lo, hi))
        assert abs(got - want) <= 1e-12 * abs(want), (lo, hi, got, want)


def test_noise_spectra_closed_form():
    """Initial truncated-Wigner state: n_m(k) = 0 and S_perp(k) = 2 (n + 1/(2 dx^d))
    (flat in k, as the paper's initial structure factor), within statistical errors."""
    shape, dx, n, ntraj = (32, 32), 0.5, 1.0, 8
    d = 2
    psis = []
    for t in range(ntraj):
        eta = tw_noise(shape, seed=77, traj=t, noise_per_mode=0.5, dx=dx)
        eta[1] += math.sqrt(n)
        psis.append(eta)
    psi = T(np.stack(psis))
    nk = O.occupation_modes(psi, dx, d)
    S = O.spin_structure_modes(psi, dx, d)
    M = ntraj * math.prod(shape)
    for m in (0, 2):
        assert abs(float(nk[:, m].mean())) < 4 * 0.5 / math.sqrt(M)
    nk0 = nk[:, 1].reshape(ntraj, -1)[:, 1:]
    assert abs(float(nk0.mean())) < 4 * 0.5 / math.sqrt(nk0.numel())
    Sexp = 2 * (n + 1 / (2 * dx ** d))
    assert abs(float(S.mean()) - Sexp) < 4 * Sexp / math.sqrt(M) * 1.5
    # flat: low and high |k| halves agree
    b = O.radial_bins(shape)
    lo = S[:, b <= 8].mean()
    hi = S[:, b > 8].mean()
    assert abs(float(lo - hi)) < 0.1 * Sexp


def test_q_ramp_piecewise_linear():
    knots = np.array([2.0, 1.0, 0.5, 0.5])
    q = O.q_piecewise_linear(knots, t_end=3.0)
    assert float(q(0.0)) == 2.0 and float(q(-1.0)) == 2.0 and float(q(5.0)) == 0.5
    assert abs(float(q(0.5)) - 1.5) < 1e-15
    assert abs(float(q(1.25)) - 0.875) < 1e-15


def test_gradient_matches_finite_differences():
    """Autograd of the oracle (the adjoint oracle) against central finite differences of
    the forward, for the q knots and for the initial field."""
    shape, dx, d = (16, 16), 1.0, 2
    psi0 = T(W.random_field(shape, 2, seed=12, scale=0.6))
    knots = torch.tensor([0.2, 0.12, 0.05], dtype=torch.float64, requires_grad=True)
    dt, nst = 0.05, 12
    tend = dt * nst

    def loss_of(kn, p0):
        qf = O.q_piecewise_linear(kn, tend)
        p = O.propagate(p0, dt, nst, 1.0, -0.1, qf, dx, d)
        return O.sf_band_loss(p, dx, d, 0.2, 1.2)

    p0 = psi0.clone().requires_grad_(True)
    L = loss_of(knots, p0)
    gk, gp = torch.autograd.grad(L, (knots, p0))
    h = 1e-5
    for i in range(3):
        kp = knots.detach().clone(); kp[i] += h
        km = knots.detach().clone(); km[i] -= h
        fd = (float(loss_of(kp, psi0)) - float(loss_of(km, psi0))) / (2 * h)
        assert abs(fd - float(gk[i])) < 1e-6 * max(1.0, abs(fd))
    # field gradient: torch convention grad = dL/dRe + i dL/dIm
    for idx in [(0, 1, 3, 4), (1, 0, 7, 2), (1, 2, 0, 15)]:
        for unit in (1.0, 1j):
            pp = psi0.clone(); pp[idx] += h * unit
            pm = psi0.clone(); pm[idx] -= h * unit
            fd = (float(loss_of(knots.detach(), pp)) - float(loss_of(knots.detach(), pm))) / (2 * h)
            an = float(gp[idx].real) if unit == 1.0 else float(gp[idx].imag)
            assert abs(fd - an) < 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------- rotation integrator

def test_rotation_operator_is_the_gpe_interaction():
    """c0 rho + c1 F.f + q f_z^2 applied to psi equals the bracket of Eq. (GPE) without
    the kinetic term (written here from the equation's matrix)."""
    g = np.random.default_rng(2)
    p = g.normal(size=3) + 1j * g.normal(size=3)
    c0, c1, q = 0.8, -0.3, 0.21
    p1, p0, pm = p
    n1, n0, nm = abs(p) ** 2
    rho = n1 + n0 + nm
    M = np.array([[-2 * nm, np.conj(pm) * p0, 0], [pm * np.conj(p0), -n0 - q / c1, np.conj(p0) * p1],
                  [0, p0 * np.conj(p1), -2 * n1]])
    gpe = (q + (c0 + c1) * rho) * p + c1 * M @ p
    Fz = n1 - nm
    Fp = math.sqrt(2) * (np.conj(p1) * p0 + np.conj(p0) * pm)
    Ff = np.array(O.spin_dot_f(torch.tensor(Fz), torch.tensor(Fp), *[torch.tensor(x) for x in p]))
    rot = c0 * rho * p + c1 * Ff + q * np.array([p1, 0, pm])
    np.testing.assert_allclose(rot, gpe, atol=1e-13)


def test_rotation_step_is_exact_flow_and_conserves_spin():
    """The rotation step equals expm of -i tau (c0 rho + c1 F.f) (scipy), keeps F and rho."""
    g = np.random.default_rng(4)
    p = g.normal(size=3) + 1j * g.normal(size=3)
    c0, c1, tau = 0.9, -0.4, 0.7
    t = torch.as_tensor(p.reshape(3, 1))
    out = O.rotation_interaction(t, tau, c0, c1, 1).numpy().ravel()
    n = abs(p) ** 2
    Fz = n[0] - n[2]
    Fp = math.sqrt(2) * (np.conj(p[0]) * p[1] + np.conj(p[1]) * p[2])
    r2 = math.sqrt(2)
    Ff = np.array([[Fz, np.conj(Fp) / r2, 0], [Fp / r2, 0, np.conj(Fp) / r2], [0, Fp / r2, -Fz]])
    ref = scipy.linalg.expm(-1j * tau * (c0 * n.sum() * np.eye(3) + c1 * Ff)) @ p
    np.testing.assert_allclose(out, ref, atol=1e-13)
    n2 = abs(out) ** 2
    assert abs(n2.sum() - n.sum()) < 1e-13 and abs((n2[0] - n2[2]) - Fz) < 1e-13


def test_rotation_scheme_fz_exact_and_second_order():
    """F_z is conserved to rounding by the rotation scheme (every factor commutes with the
    total F_z); the scheme is second order and agrees with the paper's scheme as dt -> 0."""
    psi = T(W.smooth_random_field((64,), 1, seed=3))
    c0, c1, q, dx = 1.0, -0.5, 0.09, 1.0
    out = O.propagate_rotation(psi, 0.05, 40, c0, c1, q, dx, 1)
    dg0 = O.diagnostics(psi, dx, c0, c1, q, 1)[0]
    dg1 = O.diagnostics(out, dx, c0, c1, q, 1)[0]
    assert abs(float((dg1[0] - dg1[2]) - (dg0[0] - dg0[2]))) < 1e-12
    ref = O.propagate(psi, 1.0 / 512, 512, c0, c1, q, dx, 1)
    errs = []
    for nst in (10, 20, 40):
        o = O.propagate_rotation(psi, 1.0 / nst, nst, c0, c1, q, dx, 1)
        errs.append(float((o - ref).abs().pow(2).sum().sqrt()))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_rotation_uniform_states():
    """Uniform ferromagnetic state psi_1 = sqrt(n): exp(-i (q + (c0 + c1) n) t) exactly;
    uniform polar state: exp(-i c0 n t)."""
    n, c0, c1, q, dt, steps = 0.8, 1.0, -0.1, 0.09, 0.02, 30
    psi = np.zeros((3, 16), complex)
    psi[0] = math.sqrt(n)
    out = O.propagate_rotation(T(psi), dt, steps, c0, c1, q, 1.0, 1).numpy()
    np.testing.assert_allclose(out[0], math.sqrt(n) * np.exp(-1j * (q + (c0 + c1) * n) * dt * steps), atol=1e-13)
    psi = np.zeros((3, 16), complex)
    psi[1] = math.sqrt(n)
    out = O.propagate_rotation(T(psi), dt, steps, c0, c1, q, 1.0, 1).numpy()
    np.testing.assert_allclose(out[1], math.sqrt(n) * np.exp(-1j * c0 * n * dt * steps), atol=1e-13)
