"""Scaling analysis of ensemble spectra (host side, numpy/scipy on accumulated spectra).

The paper characterises universal dynamics by the self-similar evolution of the
structure factor, Eq. (StructureFactor) of Sec. 2.1:

    S(t, k) = (t / t_ref)^alpha  f_s((t / t_ref)^beta  k),

with alpha = d beta in the IR where the momentum integral of S is conserved, and
beta ~ 1/4 for the coarsening of the Larmor-angle domains of the 1D spin-1 gas (Sec. 1).
Two estimators of the exponents are provided:

  * moments: k_Lambda(t) = sum_k k S / sum_k S over an IR window scales as t^-beta, and
    the window integral sum_k S as t^(alpha - beta) (1D: the modes are equally spaced);
  * collapse: alpha and beta minimising the squared log-distance between the rescaled
    spectra (t/t_ref)^-alpha S(t, k) at k' = (t/t_ref)^beta k and the reference spectrum
    S(t_ref, k'), interpolated log-log (the rescaling fit of the paper's Fig. 2).
"""
import numpy as np
import scipy.optimize


def ir_moments(k, S, kmax, kmin=0.0):
    """First moment and integral of S over kmin < k <= kmax for each time.

    k: (nk,) bin centres; S: (nt, nk).  Returns (k_lambda (nt,), integral (nt,))."""
    k = np.asarray(k, dtype=np.float64)
    S = np.atleast_2d(np.asarray(S, dtype=np.float64))
    m = (k > kmin) & (k <= kmax)
    tot = S[:, m].sum(axis=1)
    return (S[:, m] * k[m]).sum(axis=1) / tot, tot


def fit_power(t, y):
    """Least-squares slope and intercept of log y against log t."""
    slope, icpt = np.polyfit(np.log(np.asarray(t, dtype=np.float64)), np.log(np.asarray(y, dtype=np.float64)), 1)
    return float(slope), float(icpt)


def moment_exponents(t, k, S, kmax, kmin=0.0):
    """beta = -d log k_Lambda / d log t and alpha = beta + d log(sum S) / d log t."""
    kl, tot = ir_moments(k, S, kmax, kmin)
    beta = -fit_power(t, kl)[0]
    alpha = beta + fit_power(t, tot)[0]
    return alpha, beta


def collapse_residual(params, t, k, S, i_ref, kmax, kmin=0.0):
    """Mean squared log-distance of the rescaled spectra from the reference spectrum."""
    alpha, beta = params
    k = np.asarray(k, dtype=np.float64)
    sel = (k > kmin) & (k <= kmax) & (S[i_ref] > 0)
    lx = np.log(k[sel])
    ly = np.log(S[i_ref][sel])
    res = []
    for i in range(len(t)):
        if i == i_ref:
            continue
        s = t[i] / t[i_ref]
        kk = k * s ** beta
        ok = (k > kmin) & (S[i] > 0) & (kk > k[sel][0]) & (kk < k[sel][-1])
        if not np.any(ok):
            continue
        ref = np.interp(np.log(kk[ok]), lx, ly)
        res.append(np.log(S[i][ok] * s ** -alpha) - ref)
    if not res:
        return np.inf
    r = np.concatenate(res)
    return float(np.mean(r * r))


def collapse_exponents(t, k, S, t_ref, kmax, kmin=0.0, guess=(0.25, 0.25)):
    """(alpha, beta, residual) of the best rescaling collapse onto S(t_ref, k)."""
    t = np.asarray(t, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    i_ref = int(np.argmin(np.abs(t - t_ref)))
    out = scipy.optimize.minimize(collapse_residual, np.asarray(guess, dtype=np.float64),
                                  args=(t, k, S, i_ref, kmax, kmin), method="Nelder-Mead",
                                  options={"xatol": 1e-7, "fatol": 1e-14, "maxiter": 4000})
    return float(out.x[0]), float(out.x[1]), float(out.fun)
