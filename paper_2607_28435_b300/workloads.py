"""Seeded synthetic pricing problems.

This module only describes and draws problem parameters; it holds none of the
pricing arithmetic (no characteristic function, grid or transform), so both the
CUDA path and the CPU oracle can take their inputs from it.

A problem is the statement of Sec. 2.1 of the paper: a characteristic-function
model with its parameters, spot S0, rate r, maturity T, damping alpha
(Eq. damping_moment_condition), frequency spacing eta, grid exponent n
(M = 2^n points), a truncation tolerance, and the quadrature rule.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

# model identifiers (same values as the C enum sfft_model)
GBM, HESTON, MERTON, VG = 0, 1, 2, 3
MODEL_NAMES = {GBM: "gbm", HESTON: "heston", MERTON: "merton", VG: "vg"}
# quadrature identifiers (same values as the C enum sfft_quad)
SIMPSON_CM99, RECT_SYM = 0, 1

# parameter slots per model (p[0..]):
#   GBM    (sigma,)
#   HESTON (kappa, theta, sigma_v, rho, v0)
#   MERTON (sigma, lam, mu_j, delta_j)
#   VG     (sigma, nu, theta)
PARAM_NAMES = {
    GBM: ("sigma",),
    HESTON: ("kappa", "theta", "sigma_v", "rho", "v0"),
    MERTON: ("sigma", "lam", "mu_j", "delta_j"),
    VG: ("sigma", "nu", "theta"),
}


@dataclasses.dataclass
class Problem:
    model: int
    p: tuple
    S0: float = 100.0
    r: float = 0.05
    T: float = 1.0
    alpha: float = 1.5
    eta: float = 0.25          # SIMPSON_CM99: v_j = eta*j; RECT_SYM: Delta_v (<=0 -> paper grid)
    n: int = 12
    tol: float = 1e-12
    quad: int = SIMPSON_CM99
    k0: float = float("nan")   # RECT_SYM lower log-moneyness; NaN -> default centring
    max_rank: int = 0          # 0 -> library default

    def param(self, name: str) -> float:
        return float(self.p[PARAM_NAMES[self.model].index(name)])

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def config1_gbm() -> Problem:
    """Plain Carr-Madan, GBM: S0=100, r=0.05, sigma=0.2, T=1, alpha=1.5,
    eta=0.25, N=2^12, Simpson weights."""
    return Problem(GBM, (0.2,), S0=100.0, r=0.05, T=1.0, alpha=1.5, eta=0.25,
                   n=12, quad=SIMPSON_CM99)


HESTON_CFG2 = (1.5768, 0.0398, 0.5751, -0.5711, 0.0175)


def config2_heston(n: int, tol: float = 1e-12) -> Problem:
    """Single Heston instance: S0=100, r=0.025, T=1, kappa=1.5768,
    theta=0.0398, sigma_v=0.5751, rho=-0.5711, v0=0.0175, alpha=1.5,
    eta=0.25, tol 1e-12, n in 16..40."""
    return Problem(HESTON, HESTON_CFG2, S0=100.0, r=0.025, T=1.0, alpha=1.5,
                   eta=0.25, n=n, tol=tol, quad=SIMPSON_CM99)


def paper_grid_bs(n: int) -> Problem:
    """The paper's experimental grid (Sec. 4): Black-Scholes S0=100, r=0.05,
    sigma=0.3, T=0.5, alpha=2.5, N=2^(n-1), Delta_k=N^(-1/2),
    b=log S0 - N Delta_k/2, Delta_v = pi/(N Delta_k)."""
    return Problem(GBM, (0.3,), S0=100.0, r=0.05, T=0.5, alpha=2.5, eta=0.0,
                   n=n, quad=RECT_SYM)


CONFIG3_SEED = 260728435
CONFIG3_RANGES = {
    HESTON: [(0.5, 5.0), (0.01, 0.1), (0.1, 1.0), (-0.9, 0.0), (0.01, 0.1)],
    MERTON: [(0.1, 0.4), (0.0, 2.0), (-0.3, 0.1), (0.05, 0.3)],
    VG: [(0.1, 0.4), (0.05, 0.5), (-0.3, 0.0)],
}


def config3_batch(count: int = 4096, seed: int = CONFIG3_SEED, n_lo: int = 16,
                  n_hi: int = 34, tol: float = 1e-12) -> List[Problem]:
    """Mixed batch: model = i mod 3 (Heston, Merton, VG), parameters uniform
    in the configured boxes, T uniform in [0.1, 3], n uniform integer in
    [n_lo, n_hi]. Draw order per instance: model parameters, then T, then n.
    S0=100, r=0.025, alpha=1.5, eta=0.25, Simpson weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    order = (HESTON, MERTON, VG)
    out = []
    for i in range(count):
        model = order[i % 3]
        p = tuple(float(rng.uniform(lo, hi)) for lo, hi in CONFIG3_RANGES[model])
        T = float(rng.uniform(0.1, 3.0))
        n = int(rng.integers(n_lo, n_hi + 1))
        out.append(Problem(model, p, S0=100.0, r=0.025, T=T, alpha=1.5,
                           eta=0.25, n=n, tol=tol, quad=SIMPSON_CM99))
    return out


def heston_box_batch(count: int, seed: int, n: int = 16, tol: float = 1e-12) -> List[Problem]:
    """Heston-only draws from the batched box (used for the surrogate box)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        p = tuple(float(rng.uniform(lo, hi)) for lo, hi in CONFIG3_RANGES[HESTON])
        T = float(rng.uniform(0.1, 3.0))
        out.append(Problem(HESTON, p, S0=100.0, r=0.025, T=T, alpha=1.5,
                           eta=0.25, n=n, tol=tol, quad=SIMPSON_CM99))
    return out


def strike_set(l_begin: int, stride: int, q: int) -> np.ndarray:
    """Grid indices l_begin + i*stride, i in [0, q)."""
    return l_begin + stride * np.arange(q, dtype=np.int64)


# surrogate box: the Heston box of the mixed batch, r, T and log-moneyness
SURROGATE_NAMES = ("kappa", "theta", "sigma_v", "rho", "v0", "r", "T", "k")
SURROGATE_LO = tuple(lo for lo, _ in CONFIG3_RANGES[HESTON]) + (0.0, 0.1, -1.5)
SURROGATE_HI = tuple(hi for _, hi in CONFIG3_RANGES[HESTON]) + (0.05, 3.0, 1.5)


def heston_surrogate_batch(count: int, seed: int, n: int = 16, tol: float = 1e-12,
                           lo=SURROGATE_LO, hi=SURROGATE_HI) -> List[Problem]:
    """Heston instances with parameters, r and T uniform in [lo, hi] (the
    first seven coordinates of the surrogate box). Draw order per instance:
    the five model parameters, r, T."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        v = [float(rng.uniform(lo[i], hi[i])) for i in range(7)]
        out.append(Problem(HESTON, tuple(v[:5]), S0=100.0, r=v[5], T=v[6], alpha=1.5,
                           eta=0.25, n=n, tol=tol, quad=SIMPSON_CM99))
    return out
