"""Pins of the surrogate's FP64 reference (oracle/mlp.py) that need no GPU:
closed-form GELU values, central finite differences of the loss for every
weight and bias of a small network, Adam's first step in closed form, and
bfloat16 rounding at exactly representable, halfway and tie cases."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_form():
    # GELU(z) = z Phi(z); Phi(1) and phi(1) from their definitions
    phi1 = 0.5 * (1.0 + math.erf(1.0 / math.sqrt(2.0)))
    dens1 = math.exp(-0.5) / math.sqrt(2.0 * math.pi)
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) <= 1e-15
    assert abs(mlp.gelu(-1.0) + 0.15865525393145707) <= 1e-15
    assert abs(mlp.gelu(1.0) - phi1) <= 1e-16
    assert mlp.gelu_grad(0.0) == 0.5
    assert abs(mlp.gelu_grad(1.0) - (phi1 + dens1)) <= 1e-15
    # tails: GELU -> identity for large z, -> 0 for very negative z
    assert abs(mlp.gelu(8.0) - 8.0) <= 1e-12
    assert abs(mlp.gelu(-8.0)) <= 1e-12


def _net(widths, seed):
    rng = np.random.default_rng(seed)
    W = [rng.standard_normal((widths[l + 1], widths[l])) * 0.7 for l in range(len(widths) - 1)]
    b = [rng.standard_normal(widths[l + 1]) * 0.3 for l in range(len(widths) - 1)]
    return W, b


def test_backward_matches_central_differences():
    W, b = _net((3, 5, 4, 1), 1)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((7, 3))
    t = rng.standard_normal(7)
    dW, db, _ = mlp.backward(W, b, x, t)
    h = 1e-6
    for params, grads in ((W, dW), (b, db)):
        for P, G in zip(params, grads):
            for idx in np.ndindex(P.shape):
                old = P[idx]
                P[idx] = old + h
                fp = mlp.loss(W, b, x, t)
                P[idx] = old - h
                fm = mlp.loss(W, b, x, t)
                P[idx] = old
                fd = (fp - fm) / (2 * h)
                assert abs(fd - G[idx]) <= 1e-8 * (1.0 + abs(G[idx])), (idx, fd, G[idx])


def test_backward_of_a_linear_network_is_least_squares_gradient():
    # one layer: y = x w + b, so dL/dw = 2/B x^T (y - t), dL/db = 2/B sum (y - t)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((9, 4))
    t = rng.standard_normal(9)
    W = [rng.standard_normal((1, 4))]
    b = [rng.standard_normal(1)]
    dW, db, _ = mlp.backward(W, b, x, t)
    r = x @ W[0][0] + b[0][0] - t
    assert np.allclose(dW[0][0], 2.0 / 9 * x.T @ r, rtol=0, atol=1e-14)
    assert abs(db[0][0] - 2.0 / 9 * r.sum()) <= 1e-14


def test_adam_first_step_closed_form():
    # step 1: m_hat = g, v_hat = g^2, so p1 = p0 - lr g / (|g| + eps)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(6)
    g = rng.standard_normal(6)
    m, v = np.zeros(6), np.zeros(6)
    p0 = p.copy()
    mlp.adam_step(p, g, m, v, 1, 1e-3, 0.9, 0.999, 1e-8)
    assert np.allclose(p, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_rounding_cases():
    # bfloat16 keeps 7 fraction bits: spacing 2^-7 just above 1
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, math.pi, 1.0 + 2.0 ** -7 + 2.0 ** -9],
                    dtype=np.float32)
    want = [1.0, 1.0, 1.0 + 2.0 ** -6, -2.5, 3.140625, 1.0 + 2.0 ** -7]
    assert list(mlp.bf16_round(vals)) == want


def test_bf16_pair_encoding():
    # hi is the nearest bfloat16, lo the nearest bfloat16 of the float32
    # remainder: values a bfloat16 holds have lo = 0; 1 + 2^-10 splits into
    # 1 and 2^-10 exactly; in general hi + lo is within 2^-16 relative of x
    x = np.array([1.0, -2.5, 1.0 + 2.0 ** -10, 0.1, -0.7, 3e-3], dtype=np.float32)
    pair = mlp.bf16_pair(x)
    assert pair[0] == 1.0 and pair[1] == -2.5
    assert pair[2] == 1.0 + 2.0 ** -10
    assert np.all(np.abs(pair - x.astype(np.float64)) <= 2.0 ** -16 * np.abs(x))
    hi = mlp.bf16_round(x)
    assert np.all(np.abs(pair - hi) <= 2.0 ** -8 * np.abs(x))


def test_bf16_network_rounds_hidden_activations_and_tracks_exact_gradients():
    W, b = _net((5, 12, 9, 1), 8)
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, size=(11, 5)).astype(np.float32)
    t = rng.standard_normal(11)
    y, zs, hs = mlp.forward(W, b, x, act_bf16=True)
    # every hidden activation fed to a product is a bfloat16 value: GELU(z) rounded
    for l in (1, 2):
        h = hs[l]
        assert np.array_equal(h, mlp.bf16_round(h))
        assert np.all(np.abs(h - mlp.gelu(zs[l - 1])) <= 2.0 ** -8 * np.abs(mlp.gelu(zs[l - 1])) + 1e-300)
    # the output is linear in the last activations
    assert np.allclose(y, hs[2] @ W[2][0] + b[2][0], rtol=0, atol=1e-13)
    # with the rounding passed through, the gradients differ from the exact
    # float64 network's only by the bfloat16 steps (a few parts in 10^3),
    # not by a dropped or transposed term
    dW, db, _ = mlp.backward(W, b, x, t, act_bf16=True)
    dW0, db0, _ = mlp.backward(W, b, x.astype(np.float64), t)
    for a, c in zip(dW + db, dW0 + db0):
        assert np.max(np.abs(a - c)) <= 2e-2 * np.max(np.abs(c)) + 1e-12
