"""Exponent estimators of the scaling analysis on synthetic spectra that obey
Eq. (StructureFactor) exactly, S(t, k) = (t/t_ref)^alpha f_s((t/t_ref)^beta k) (no GPU)."""
import numpy as np
import pytest

from paper_2310_03636_gb300 import scaling


def synthetic(alpha, beta, noise=0.0, seed=0, p=1.2):
    t = np.array([100.0, 200.0, 400.0, 800.0, 1600.0, 3200.0])
    k = 2 * np.pi * np.arange(1, 2049) / 4096.0
    k0 = 0.08

    def f(u):   # plateau in the IR, power-law fall-off k^-2p above k0
        return 1.0 / (1.0 + (u / k0) ** 2) ** p

    S = np.stack([(ti / 400.0) ** alpha * f((ti / 400.0) ** beta * k) for ti in t])
    if noise:
        S = S * np.exp(noise * np.random.default_rng(seed).standard_normal(S.shape))
    return t, k, S


@pytest.mark.parametrize("alpha,beta", [(0.25, 0.25), (0.27, 0.25), (0.5, 0.5), (-0.1, -0.2)])
def test_collapse_recovers_exponents(alpha, beta):
    t, k, S = synthetic(alpha, beta)
    a, b, r = scaling.collapse_exponents(t, k, S, t_ref=400.0, kmax=0.6, guess=(0.0, 0.0))
    assert abs(a - alpha) < 1e-4 and abs(b - beta) < 1e-4 and r < 1e-8


def test_collapse_with_noise():
    t, k, S = synthetic(0.27, 0.25, noise=0.03, seed=4)
    a, b, _ = scaling.collapse_exponents(t, k, S, t_ref=400.0, kmax=0.6)
    assert abs(a - 0.27) < 0.02 and abs(b - 0.25) < 0.02


def test_moment_exponents():
    """The first moment over the whole spectrum scales as t^-beta when the window holds
    (nearly) all of f_s, here a k^-6 fall-off; the integral as t^(alpha - beta)."""
    t, k, S = synthetic(0.27, 0.25, p=3.0)
    a, b = scaling.moment_exponents(t, k, S, kmax=np.pi)
    assert abs(b - 0.25) < 0.02 and abs(a - 0.27) < 0.02


def test_fit_power_exact():
    t = np.array([1.0, 2.0, 4.0, 8.0])
    s, c = scaling.fit_power(t, 3.0 * t ** -0.4)
    assert abs(s + 0.4) < 1e-12 and abs(c - np.log(3.0)) < 1e-12
