"""Characteristic functions and the Carr-Madan transform psi -- oracle (test
infrastructure only).

All functions use log-moneyness: X = log(S_T / S0), phi1(u) = E[exp(i u X)]
under the risk-neutral measure, so that phi(u) of Eq. characteristic_function
equals exp(i u log S0) * phi1(u). Complex u is allowed everywhere (Eq. psi
evaluates phi at v - i(alpha+1)).

The paper gives the Black-Scholes model (Sec. 2) and names Heston, Merton and
Variance-Gamma (Sec. 2, Sec. 1) without formulas; their characteristic functions
are the standard published ones:
  * Black-Scholes: from the solution S_t = S0 exp(sigma W_t + (r - sigma^2/2) t).
  * Heston (1993) in the "little trap" form of Albrecher, Mayer, Schoutens and
    Tistaert (2007), principal square root.
  * Merton (1976) jump diffusion with log-normal jumps, compensated drift.
  * Variance Gamma (Madan, Carr and Chang 1998) with the martingale
    correction omega.
"""
from __future__ import annotations

import numpy as np

GBM, HESTON, MERTON, VG = 0, 1, 2, 3


def phi1(model: int, p, r: float, T: float, u):
    """phi1(u) = E[exp(i u log(S_T/S0))] for complex array u."""
    u = np.asarray(u, dtype=np.complex128)
    iu = 1j * u
    if model == GBM:
        (sigma,) = p[:1]
        return np.exp(iu * (r - 0.5 * sigma * sigma) * T - 0.5 * sigma * sigma * u * u * T)
    if model == HESTON:
        kappa, theta, sv, rho, v0 = p[:5]
        b = kappa - rho * sv * iu
        d = np.sqrt(b * b + sv * sv * (iu + u * u))
        g = (b - d) / (b + d)
        e = np.exp(-d * T)
        C = kappa * theta / (sv * sv) * ((b - d) * T - 2.0 * np.log((1.0 - g * e) / (1.0 - g)))
        D = (b - d) / (sv * sv) * (1.0 - e) / (1.0 - g * e)
        return np.exp(iu * r * T + C + D * v0)
    if model == MERTON:
        sigma, lam, muj, dj = p[:4]
        kbar = np.exp(muj + 0.5 * dj * dj) - 1.0
        drift = iu * (r - 0.5 * sigma * sigma - lam * kbar) * T
        diff = -0.5 * sigma * sigma * u * u * T
        jump = lam * T * (np.exp(iu * muj - 0.5 * dj * dj * u * u) - 1.0)
        return np.exp(drift + diff + jump)
    if model == VG:
        sigma, nu, theta = p[:3]
        omega = np.log(1.0 - theta * nu - 0.5 * sigma * sigma * nu) / nu
        base = 1.0 - iu * theta * nu + 0.5 * sigma * sigma * nu * u * u
        return np.exp(iu * (r + omega) * T - (T / nu) * np.log(base))
    raise ValueError(f"unknown model {model}")


def psi1(model: int, p, r: float, T: float, alpha: float, v):
    """Eq. psi in log-moneyness:
    psi1(v) = exp(-rT) phi1(v - i(alpha+1)) / ((alpha + iv)(alpha + 1 + iv))."""
    v = np.asarray(v, dtype=np.float64)
    num = phi1(model, p, r, T, v - 1j * (alpha + 1.0))
    den = (alpha + 1j * v) * (alpha + 1.0 + 1j * v)
    return np.exp(-r * T) * num / den
