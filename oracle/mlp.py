"""Test infrastructure: the FP64 reference of the price surrogate (a plain
multilayer perceptron fitted to SFFT prices; no counterpart in the paper,
which builds the pricing map itself as a tensor network, Sec. 3).

Only the tests, the package's smoke check and the bench's CPU leg may import
this module. It is written for checking, not speed.

Network: h_0 = x; z_l = W_l h_{l-1} + b_l (l = 1..L); h_l = GELU(z_l) for
l < L; the output y = z_L is linear. GELU(z) = z Phi(z) with the standard
normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2, so GELU'(z) = Phi(z) + z phi(z).
Loss: mean over the batch of (y - t)^2. Gradients by the chain rule, layer by
layer from the output (reverse-mode differentiation of the above).

Tensor-core arithmetic (act_bf16=True): the products take bfloat16 operands,
so the network as evaluated there feeds the inputs as the pair hi + lo (hi the
nearest bfloat16 of the float32 input, lo the nearest bfloat16 of the float32
remainder) and rounds every hidden activation h_l to the nearest bfloat16
before the next product. The backward pass differentiates that network with
the rounding passed through unchanged (its derivative taken as 1).

Parity: pinned by central finite differences of the loss (every weight and
bias of a small network) and by closed-form GELU values; see
tests/test_mlp_oracle.py.
"""
import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def phi_cdf(z):
    """Standard normal CDF, elementwise, through erf."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + np.vectorize(math.erf)(z / SQRT2))


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return z * phi_cdf(z)


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    return phi_cdf(z) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def bf16_pair(x):
    """hi + lo for float32 inputs x: hi = bfloat16(x), lo = bfloat16(x - hi),
    the difference taken in float32 (where it is exact)."""
    xf = np.asarray(x, dtype=np.float32)
    hi = bf16_round(xf)
    lo = bf16_round(xf - hi.astype(np.float32))
    return hi + lo


def forward(weights, biases, x, act_bf16=False):
    """x: (B, width[0]). weights[l]: (width[l+1], width[l]); biases[l]:
    (width[l+1],). Returns (y of shape (B,), the pre-activations z_l and the
    layer inputs h_{l-1}, both per layer). act_bf16: the tensor-core
    arithmetic described above."""
    h = bf16_pair(x) if act_bf16 else np.asarray(x, dtype=np.float64)
    zs, hs = [], []
    L = len(weights)
    for l in range(L):
        hs.append(h)
        z = h @ np.asarray(weights[l], dtype=np.float64).T + np.asarray(biases[l], dtype=np.float64)
        zs.append(z)
        if l < L - 1:
            h = bf16_round(gelu(z)) if act_bf16 else gelu(z)
        else:
            h = z
    return h[:, 0], zs, hs


def loss(weights, biases, x, t, act_bf16=False):
    y, _, _ = forward(weights, biases, x, act_bf16)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward_from(weights, zs, hs, dy):
    """The chain rule from the output down, given the forward pass's
    pre-activations zs, layer inputs hs and dL/dy: (dW, db) per layer."""
    dz = np.asarray(dy, dtype=np.float64)[:, None]
    L = len(weights)
    dW = [None] * L
    db = [None] * L
    for l in range(L - 1, -1, -1):
        dW[l] = dz.T @ np.asarray(hs[l], dtype=np.float64)
        db[l] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ np.asarray(weights[l], dtype=np.float64)
            dz = dh * gelu_grad(zs[l - 1])
    return dW, db


def backward(weights, biases, x, t, act_bf16=False):
    """Gradients of the mean squared error: (dW per layer, db per layer,
    dL/dy per sample)."""
    y, zs, hs = forward(weights, biases, x, act_bf16)
    B = y.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B
    dW, db = backward_from(weights, zs, hs, dy)
    return dW, db, dy


def adam_step(p, g, m, v, step, lr, beta1, beta2, eps):
    """One Adam update (Kingma & Ba 2015) of p in place, with bias-corrected
    moments; m and v are updated in place too."""
    m *= beta1
    m += (1.0 - beta1) * g
    v *= beta2
    v += (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p -= lr * mh / (np.sqrt(vh) + eps)
    return p


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64: the weights the kernels multiply with."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
