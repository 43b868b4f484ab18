"""The discrete Carr-Madan sum, written out plainly -- oracle (test
infrastructure only).

Everything is in log-moneyness k' = log(K/S0); a call price is
C(K) = S0 * C1(k'), with C1 built from phi1 (cf.py). This reproduces the
paper's absolute-log-strike discretisation exactly (the S0 phases cancel) and
makes every grid phase an exact fraction of a turn.

Two quadrature rules:

SIMPSON_CM99 (the "higher-order quadrature weights" the paper allows after
Eq. discretization_dft; Carr and Madan 1999):
    v_j = eta*j, lambda = 2*pi/(M*eta), b = pi/eta, k'_u = -b + lambda*u,
    x_j = exp(i*b*v_j) * w_j * eta * psi1(v_j) = (-1)^j w_j eta psi1(eta j),
    w_0 = 1/3, w_odd = 4/3, w_even>0 = 2/3,
    C1(k'_u) = Re[ exp(-alpha k'_u)/pi * sum_j exp(-2 pi i j u/M) x_j ]
             = exp(-alpha k'_u)/pi * sqrt(M) * Re(y_u)   with y of Eq. dft.

RECT_SYM (Eqs. Ck_from_psi, discretization, x, discretization_dft; the grid of
Sec. 4 when eta <= 0):
    N = M/2, Delta_v = eta (or pi/sqrt(N) on the paper grid),
    Delta_k = pi/(N Delta_v), k'_0 = -N Delta_k/2 (literal reading of
    b = log S0 - N Delta_k/2), k'_l = k'_0 + l Delta_k.
    Delta_v*k'_0 = -pi/2, so Eq. x becomes
    x_j = i^j (-i)^N psi1(Delta_v (j - N)), and
    C1(k'_l) = Re[ exp(-alpha k'_l)/(2 pi) Delta_v (-1)^l sqrt(M) y_l ].
    The paper does not say to take the real part; the symmetric sum has one
    unpaired term, so the result carries a small imaginary part, and the QFT
    readout of Eq. qft_phase_assumption imposes the same positive phase.

The unitary DFT y_l = M^{-1/2} sum_j x_j exp(-2 pi i j l / M) (Eq. dft) is
computed three independent ways: an explicit matrix (small M), an iterative
radix-2 FFT, and a direct sum over a list of j at requested l whose phase
(j*l mod M) is taken in exact integer arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

from . import cf

SIMPSON_CM99, RECT_SYM = 0, 1


# ----------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------
def grid(prob):
    """Scalars of the discretisation. Returns a dict with M, the frequency
    step dv, the log-strike step dk, the lowest log-moneyness k0, and for
    RECT_SYM the half size N."""
    n = int(prob.n)
    M = 1 << n
    if prob.quad == SIMPSON_CM99:
        eta = float(prob.eta)
        dk = 2.0 * math.pi / (M * eta)
        return dict(M=M, n=n, dv=eta, dk=dk, k0=-math.pi / eta, N=None)
    if prob.quad == RECT_SYM:
        N = M // 2
        dv = float(prob.eta) if prob.eta > 0 else math.pi / math.sqrt(N)
        dk = math.pi / (N * dv)
        return dict(M=M, n=n, dv=dv, dk=dk, k0=-N * dk / 2.0, N=N)
    raise ValueError("unknown quadrature")


def log_moneyness(prob, u):
    g = grid(prob)
    return g["k0"] + g["dk"] * np.asarray(u, dtype=np.float64)


def simpson_weight(j):
    j = np.asarray(j, dtype=np.int64)
    w = np.where(j % 2 == 1, 4.0 / 3.0, 2.0 / 3.0)
    return np.where(j == 0, 1.0 / 3.0, w)


def integrand(prob, j):
    """x_j for an int64 array of indices j in [0, M)."""
    j = np.asarray(j, dtype=np.int64)
    g = grid(prob)
    if prob.quad == SIMPSON_CM99:
        v = g["dv"] * j.astype(np.float64)
        sign = np.where(j % 2 == 0, 1.0, -1.0)
        psi = cf.psi1(prob.model, prob.p, prob.r, prob.T, prob.alpha, v)
        return sign * simpson_weight(j) * g["dv"] * psi
    N = g["N"]
    v = g["dv"] * (j - N).astype(np.float64)
    i_pow = np.array([1, 1j, -1, -1j])[j % 4]
    mi_pow_N = np.array([1, -1j, -1, 1j])[N % 4]
    return i_pow * mi_pow_N * cf.psi1(prob.model, prob.p, prob.r, prob.T, prob.alpha, v)


def price_scale(prob, u):
    """The real factor multiplying Re(phase_u * y_u) in the price, and the
    phase_u, for output indices u: price = S0 * scale * Re(phase * y)."""
    g = grid(prob)
    u = np.asarray(u, dtype=np.int64)
    kp = log_moneyness(prob, u)
    sqM = math.sqrt(g["M"])
    if prob.quad == SIMPSON_CM99:
        return np.exp(-prob.alpha * kp) / math.pi * sqM, np.ones(u.shape)
    phase = np.where(u % 2 == 0, 1.0, -1.0)
    return np.exp(-prob.alpha * kp) * g["dv"] / (2.0 * math.pi) * sqM, phase


def prices_from_y(prob, u, y):
    """Eq. discretization_dft (RECT_SYM) or its Simpson analogue: call prices
    in currency units and the absolute log-strikes log K."""
    scale, phase = price_scale(prob, u)
    c = prob.S0 * scale * np.real(phase * np.asarray(y))
    logk = math.log(prob.S0) + log_moneyness(prob, u)
    return c, logk


def prices_qft_readout(prob, u, y):
    """Eq. qft_observable_price with exact probabilities: the QFT route reads
    |y_l| (sqrt of p_l times ||x||), i.e. it imposes the positive phase of
    Eq. qft_phase_assumption instead of taking the real part."""
    scale, _ = price_scale(prob, u)
    return prob.S0 * scale * np.abs(np.asarray(y))


# ----------------------------------------------------------------------------
# the unitary DFT of Eq. dft, three routes
# ----------------------------------------------------------------------------
def _unit_phase(t, M):
    """exp(-2 pi i t / M) for integer t in [0, M)."""
    ang = (2.0 * math.pi / M) * np.asarray(t, dtype=np.float64)
    return np.cos(ang) - 1j * np.sin(ang)


def dft_direct(x):
    """y = F x / sqrt(M) with the explicit matrix F[l, j] = exp(-2 pi i jl/M)."""
    x = np.asarray(x, dtype=np.complex128)
    M = x.shape[0]
    idx = np.arange(M, dtype=np.int64)
    y = np.empty(M, dtype=np.complex128)
    for l0 in range(0, M, 256):
        ls = idx[l0:l0 + 256]
        F = _unit_phase((ls[:, None] * idx[None, :]) % M, M)
        y[l0:l0 + 256] = F @ x
    return y / math.sqrt(M)


def fft_radix2(x):
    """Iterative decimation-in-time radix-2 Cooley-Tukey FFT (bit-reversed
    input order, butterflies of doubling span), scaled by M^{-1/2}."""
    a = np.asarray(x, dtype=np.complex128).copy()
    M = a.shape[0]
    n = M.bit_length() - 1
    assert 1 << n == M
    # bit-reversal permutation of the input
    j = np.arange(M, dtype=np.int64)
    rev = np.zeros(M, dtype=np.int64)
    for b in range(n):
        rev |= ((j >> b) & 1) << (n - 1 - b)
    a = a[rev]
    half = 1
    while half < M:
        span = 2 * half
        w = _unit_phase(np.arange(half, dtype=np.int64) * (M // span), M)
        a = a.reshape(M // span, span)
        top = a[:, :half].copy()
        bot = a[:, half:] * w[None, :]
        a[:, :half] = top + bot
        a[:, half:] = top - bot
        a = a.reshape(M)
        half = span
    return a / math.sqrt(M)


def sparse_sum(j, xj, u, n, chunk=1 << 18):
    """y_u = M^{-1/2} sum_k x_{j_k} exp(-2 pi i (j_k u mod M)/M) for the listed
    indices j (int64) and requested outputs u. The product j*u is formed in
    uint64, whose wrap-around is exact modulo 2^64 and therefore modulo
    M = 2^n."""
    M = 1 << n
    j = np.asarray(j, dtype=np.uint64)
    xj = np.asarray(xj, dtype=np.complex128)
    u = np.asarray(u, dtype=np.uint64)
    mask = np.uint64(M - 1)
    y = np.zeros(u.shape[0], dtype=np.complex128)
    for s in range(0, j.shape[0], chunk):
        jj = j[s:s + chunk]
        xx = xj[s:s + chunk]
        for k in range(u.shape[0]):
            t = (jj * u[k]) & mask
            y[k] += np.dot(xx, _unit_phase(t, M))
    return y / math.sqrt(M)


# ----------------------------------------------------------------------------
# tail of the integrand (how far the direct sum must run)
# ----------------------------------------------------------------------------
def psi_envelope(prob, v):
    """A decreasing upper bound on |psi1(v)| for v >= 0 (GBM, Merton, VG),
    from |phi1(v - ip)| <= |exp(...)| of each exponent's real part, p = alpha+1,
    and |alpha + iv| |alpha + 1 + iv| >= sqrt((alpha^2+v^2)((alpha+1)^2+v^2))."""
    v = np.asarray(v, dtype=np.float64)
    a, r, T = prob.alpha, prob.r, prob.T
    p = a + 1.0
    den = np.sqrt((a * a + v * v) * (p * p + v * v))
    if prob.model == cf.GBM:
        (s,) = prob.p[:1]
        lg = p * (r - 0.5 * s * s) * T - 0.5 * s * s * T * (v * v - p * p)
    elif prob.model == cf.MERTON:
        s, lam, mu, dj = prob.p[:4]
        kbar = math.exp(mu + 0.5 * dj * dj) - 1.0
        jmod = np.exp(p * mu - 0.5 * dj * dj * (v * v - p * p))
        lg = (p * (r - 0.5 * s * s - lam * kbar) * T - 0.5 * s * s * T * (v * v - p * p)
              + lam * T * (jmod + 1.0))
    elif prob.model == cf.VG:
        s, nu, th = prob.p[:3]
        omega = math.log(1.0 - th * nu - 0.5 * s * s * nu) / nu
        c0 = 1.0 - p * th * nu - 0.5 * s * s * nu * p * p
        lg = p * (r + omega) * T - (T / nu) * np.log(c0 + 0.5 * s * s * nu * v * v)
    else:
        raise ValueError("no closed envelope for this model")
    return np.exp(-r * T) * np.exp(lg) / den


def tail_bound(prob, J):
    """Upper bound on sum_{J <= j < M} |x_j| (Simpson grid, weights <= 4/3),
    by summing the decreasing envelope over geometric blocks with its value at
    each block's left end. Heston has no closed envelope: it returns NaN."""
    g = grid(prob)
    M = g["M"]
    if J >= M:
        return 0.0
    if prob.model == cf.HESTON or prob.quad != SIMPSON_CM99:
        return float("nan")
    edges = np.unique(np.concatenate([
        np.array([J], dtype=np.float64),
        np.geomspace(max(J, 1), M, 4096),
        np.array([M], dtype=np.float64)]))
    left, right = edges[:-1], edges[1:]
    env = psi_envelope(prob, g["dv"] * np.floor(left))
    return float(4.0 / 3.0 * g["dv"] * np.sum(env * (np.ceil(right) - np.floor(left))))


def support_limit(prob, tail_tol=1e-13):
    """Smallest power of two J = 2^m (m <= n) beyond which the integrand is
    negligible for the direct sum: the closed tail bound is below tail_tol
    (GBM, Merton, VG); for Heston, whose characteristic function decays
    exponentially, the first dyadic block [2^m, 2^(m+1)) whose samples all lie
    below tail_tol * 1e-3 / 2^m, scanned on a dense grid."""
    g = grid(prob)
    n = g["n"]
    if prob.quad != SIMPSON_CM99:
        return g["M"]
    if prob.model != cf.HESTON:
        for m in range(4, n + 1):
            if tail_bound(prob, 1 << m) <= tail_tol:
                return 1 << m
        return g["M"]
    for m in range(8, n):
        blk = np.arange(1 << m, 1 << (m + 1), dtype=np.int64)
        if np.max(np.abs(integrand(prob, blk))) * (1 << m) <= tail_tol * 1e-3:
            return 1 << m
    return g["M"]


# ----------------------------------------------------------------------------
# prices
# ----------------------------------------------------------------------------
def y_full(prob, route="fft"):
    g = grid(prob)
    x = integrand(prob, np.arange(g["M"], dtype=np.int64))
    if route == "direct":
        return dft_direct(x)
    if route == "fft":
        return fft_radix2(x)
    raise ValueError(route)


def y_at(prob, u, J=None):
    """y at requested outputs u by the direct sum over j < J (default: the
    support limit)."""
    g = grid(prob)
    if J is None:
        J = support_limit(prob)
    J = min(int(J), g["M"])
    y = np.zeros(len(u), dtype=np.complex128)
    step = 1 << 20
    for s in range(0, J, step):
        j = np.arange(s, min(J, s + step), dtype=np.int64)
        y += sparse_sum(j, integrand(prob, j), u, g["n"]) * math.sqrt(g["M"])
    return y / math.sqrt(g["M"])


def prices(prob, u, route="sparse", J=None):
    """Call prices (currency) and log-strikes at grid indices u."""
    u = np.asarray(u, dtype=np.int64)
    if route == "sparse":
        y = y_at(prob, u, J)
    else:
        y = y_full(prob, route)[u]
    return prices_from_y(prob, u, y)


def strike_window(prob, lo=-1.5, hi=1.5, qmax=4096):
    """Grid indices u with lo <= k'_u <= hi, thinned by the smallest power of
    two stride that leaves at most qmax of them, the first one aligned to the
    stride. Returns (l_begin, stride, q)."""
    g = grid(prob)
    u_lo = math.ceil((lo - g["k0"]) / g["dk"] - 1e-9)
    u_hi = math.floor((hi - g["k0"]) / g["dk"] + 1e-9)
    u_lo = max(u_lo, 0)
    u_hi = min(u_hi, g["M"] - 1)
    stride = 1
    while True:
        first = -(-u_lo // stride) * stride
        q = (u_hi - first) // stride + 1 if u_hi >= first else 0
        if q <= qmax:
            return first, stride, q
        stride *= 2


# ----------------------------------------------------------------------------
# error measure
# ----------------------------------------------------------------------------
def nrmse(prob, c, logk, c_ref_fn, k_lo=50.0, k_hi=150.0):
    """Eq. error_measure: sqrt(mean((C - C_ref)^2)) / S0 over the grid strikes
    with k_lo <= K <= k_hi."""
    K = np.exp(logk)
    sel = (K >= k_lo) & (K <= k_hi)
    err = c[sel] - c_ref_fn(K[sel])
    return math.sqrt(np.mean(err * err)) / prob.S0, int(sel.sum())
