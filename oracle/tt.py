"""Tensor trains on dense numpy arrays -- oracle (test infrastructure only).

Sec. 3.1 of the paper: a TT (Eq. tt_format) is a list of cores A_k of shape
(r_{k-1}, d, r_k); a TT operator (Eq. tto_format) has cores of shape
(s_{k-1}, d_out, d_in, s_k). The quantics index of Eq. discretized_x is
j = sum_l lambda_l 2^(n-l): site 1 is the most significant bit, so a core list
contracts to a vector in C order of shape (2,)*n.

Sec. 3.2: QFT_n = R_n Q_n, where R_n is the bit-reversal permutation of the
output and Q_n, the SFFT operator, maps x to the DFT y with its output bits in
reversed site order: output site l carries bit mu_l of the output index u
with weight 2^(l-1). Densely, row index sum_l mu_l 2^(n-l) = bitrev_n(u).

TT-SVD and rounding follow Oseledets (2011): successive truncated SVDs with
per-bond threshold delta = eps * ||A||_F / sqrt(n-1).
"""
from __future__ import annotations

import math

import numpy as np


def bitrev(u, n):
    u = np.asarray(u, dtype=np.int64)
    out = np.zeros_like(u)
    for b in range(n):
        out |= ((u >> b) & 1) << (n - 1 - b)
    return out


def trunc_rank(s, delta):
    """Smallest rank k with sqrt(sum_{i>=k} s_i^2) <= delta (s descending)."""
    tail = np.sqrt(np.cumsum((s * s)[::-1]))[::-1]  # tail[i] = ||s[i:]||
    k = len(s)
    for i in range(len(s)):
        if tail[i] <= delta:
            k = i
            break
    return max(k, 1)


def tt_full(cores):
    """Contract a TT (or a TT with d>2) to a dense array of shape (d1,...,dn)."""
    v = np.ones((1, 1), dtype=np.complex128)
    dims = []
    for G in cores:
        r0, d, r1 = G.shape
        v = (v.reshape(-1, r0) @ G.reshape(r0, d * r1)).reshape(-1, r1)
        dims.append(d)
    return v.reshape(dims)


def tt_svd(A, eps):
    """TT-SVD of a dense tensor A (shape (d1,...,dn))."""
    A = np.asarray(A, dtype=np.complex128)
    dims = A.shape
    n = len(dims)
    nrm = np.linalg.norm(A)
    delta = eps * nrm / math.sqrt(max(n - 1, 1))
    cores = []
    C = A.reshape(1, -1)
    r = 1
    for k in range(n - 1):
        C = C.reshape(r * dims[k], -1)
        U, s, Vh = np.linalg.svd(C, full_matrices=False)
        rk = trunc_rank(s, delta)
        cores.append(U[:, :rk].reshape(r, dims[k], rk))
        C = s[:rk, None] * Vh[:rk]
        r = rk
    cores.append(C.reshape(r, dims[-1], 1))
    return cores


def tt_ranks(cores):
    return [1] + [G.shape[2] for G in cores]


def tt_round(cores, eps):
    """Oseledets' TT-rounding: right-to-left QR orthogonalisation, then a
    left-to-right sweep of truncated SVDs with delta = eps ||A|| / sqrt(n-1)."""
    cores = [np.array(G, dtype=np.complex128) for G in cores]
    n = len(cores)
    for k in range(n - 1, 0, -1):
        r0, d, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0, d * r1).T.conj())
        cores[k] = Q.T.conj().reshape(-1, d, r1)
        rp = cores[k - 1].shape
        cores[k - 1] = (cores[k - 1].reshape(-1, r0) @ R.T.conj()).reshape(rp[0], rp[1], -1)
    nrm = np.linalg.norm(cores[0])
    delta = eps * nrm / math.sqrt(max(n - 1, 1))
    for k in range(n - 1):
        r0, d, r1 = cores[k].shape
        U, s, Vh = np.linalg.svd(cores[k].reshape(r0 * d, r1), full_matrices=False)
        rk = trunc_rank(s, delta)
        cores[k] = U[:, :rk].reshape(r0, d, rk)
        nxt = cores[k + 1]
        cores[k + 1] = ((s[:rk, None] * Vh[:rk]) @ nxt.reshape(r1, -1)).reshape(rk, nxt.shape[1], nxt.shape[2])
    return cores


def mpo_full(cores):
    """Dense matrix of a TT operator with cores (s, 2, 2, s') indexed
    [a, mu, lam, a'] (or (s, 4, s') with phys index 2*mu + lam). Rows are the
    output bits mu_1..mu_n read most significant first, columns the input bits
    lambda_1..lambda_n read most significant first."""
    n = len(cores)
    W = [np.asarray(G, dtype=np.complex128).reshape(G.shape[0], 2, 2, G.shape[-1]) for G in cores]
    T = np.ones((1, 1, 1), dtype=np.complex128)  # (rows, cols, bond)
    for G in W:
        s0, _, _, s1 = G.shape
        T = np.einsum("xya,amlb->xmylb", T, G).reshape(T.shape[0] * 2, T.shape[1] * 2, s1)
    return T[:, :, 0]


def qft_bitrev_dense(n):
    """Q_n from its definition: the unitary DFT matrix of Eq. dft with the
    output index bit-reversed, Q[bitrev(u), j] = M^{-1/2} exp(-2 pi i j u / M)."""
    M = 1 << n
    u = np.arange(M, dtype=np.int64)
    j = np.arange(M, dtype=np.int64)
    t = (u[:, None] * j[None, :]) % M
    F = np.exp(-2j * math.pi * t / M) / math.sqrt(M)
    Q = np.empty_like(F)
    Q[bitrev(u, n)] = F
    return Q


def qft_bitrev_product_form(n):
    """Q_n written as the product over site pairs l' <= l of
    exp(-2 pi i lambda_l mu_l' 2^(l'-l-1)) (the pairs with l' > l contribute
    whole turns), times M^{-1/2}; rows/cols as in mpo_full."""
    M = 1 << n
    rows = np.arange(M, dtype=np.int64)
    cols = np.arange(M, dtype=np.int64)
    mu = [(rows >> (n - l)) & 1 for l in range(1, n + 1)]
    lam = [(cols >> (n - l)) & 1 for l in range(1, n + 1)]
    ph = np.zeros((M, M))
    for l in range(1, n + 1):
        for lp in range(1, l + 1):
            ph += np.outer(mu[lp - 1], lam[l - 1]) * 2.0 ** (lp - l - 1)
    return np.exp(-2j * math.pi * ph) / math.sqrt(M)


def rank1_exp_tt(gamma, n):
    """Rank-one TT of g(lambda) = exp(gamma * x(lambda)), x = sum lambda_l 2^-l
    (Sec. 3.3): core l holds [1, exp(gamma 2^-l)]."""
    cores = []
    for l in range(1, n + 1):
        G = np.zeros((1, 2, 1), dtype=np.complex128)
        G[0, 0, 0] = 1.0
        G[0, 1, 0] = np.exp(gamma * 2.0 ** (-l))
        cores.append(G)
    return cores


def tt_entry(cores, bits):
    """One entry of a TT: the product of the core slices selected by the
    physical indices `bits` (site 1 first)."""
    v = np.ones((1,), dtype=np.complex128)
    for G, b in zip(cores, bits):
        v = v @ np.asarray(G)[:, int(b), :]
    return complex(v[0])
