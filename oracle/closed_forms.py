"""Closed-form prices -- oracle (test infrastructure only).

* Black-Scholes call (Eq. analytic_BS) and the matching put by parity.
* Merton (1976) jump-diffusion call as the Poisson-weighted series of
  Black-Scholes prices, truncated once the Poisson weight drops below 1e-17.
"""
from __future__ import annotations

import math

import numpy as np


def norm_cdf(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * np.vectorize(math.erfc)(-x / math.sqrt(2.0))


def bs_call(S0, K, r, sigma, T):
    """Eq. analytic_BS: Phi(d1) S0 - Phi(d2) K exp(-rT)."""
    K = np.asarray(K, dtype=np.float64)
    sq = sigma * math.sqrt(T)
    d1 = (np.log(S0 / K) + (r + 0.5 * sigma * sigma) * T) / sq
    d2 = d1 - sq
    return norm_cdf(d1) * S0 - norm_cdf(d2) * K * math.exp(-r * T)


def bs_put(S0, K, r, sigma, T):
    K = np.asarray(K, dtype=np.float64)
    return bs_call(S0, K, r, sigma, T) - S0 + K * math.exp(-r * T)


def merton_call(S0, K, r, sigma, lam, muj, dj, T, wtol=1e-17):
    """sum_k exp(-lam' T)(lam' T)^k/k! * BS(S0, K, r_k, sigma_k, T) with
    kbar = exp(muj + dj^2/2) - 1, lam' = lam (1 + kbar),
    r_k = r - lam kbar + k log(1 + kbar)/T, sigma_k^2 = sigma^2 + k dj^2/T."""
    K = np.asarray(K, dtype=np.float64)
    kbar = math.exp(muj + 0.5 * dj * dj) - 1.0
    lp = lam * (1.0 + kbar)
    out = np.zeros_like(K)
    k = 0
    while True:
        w = math.exp(-lp * T + k * math.log(lp * T) - math.lgamma(k + 1)) if lp > 0 else (1.0 if k == 0 else 0.0)
        rk = r - lam * kbar + k * math.log1p(kbar) / T
        sk = math.sqrt(sigma * sigma + k * dj * dj / T)
        out += w * bs_call(S0, K, rk, sk, T)
        if k > lp * T and w < wtol:
            break
        if lp == 0:
            break
        k += 1
    return out
