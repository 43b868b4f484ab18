"""The surrogate's tensor-core forward pass (tcgen05, include/sfft_mlp.h mode
SFFT_MLP_TENSOR_CORES) against the FP64 reference of oracle/mlp.py with the
same arithmetic (bfloat16 weights, the inputs as the bfloat16 pair hi + lo,
hidden activations rounded to bfloat16).

Tolerances, from the arithmetic:
  * a layer's pre-activation z = h W^T + b from the GPU's own bfloat16 inputs
    h: float32 accumulation of K products, bounded by 2 K 2^-24 times the sum
    of the magnitudes of the terms (K <= 256);
  * a hidden activation: exactly a bfloat16 value, within the rounding of
    GELU(z) to bfloat16 (half a step, 2^-8 relative) plus the error of the
    kernel's GELU (Hastings' erf approximation, at most 1.5e-7 in erf, so
    below 1e-7 |z| in GELU, and float32 rounding);
  * end to end, against the reference's own bfloat16 chain: rounding
    decisions taken on float32 and float64 GELU values can differ where the
    two straddle a bfloat16 midpoint, each such flip moving one activation
    by one bfloat16 step (2^-8 relative), so the outputs agree to a few
    parts in 10^3 of their scale rather than to float32 precision.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft, surrogate
    build.build()
    return sfft, surrogate


def _mlp(surrogate, widths, seed, scale=0.4):
    m = surrogate.MLP(widths, seed=seed, tensor_cores=True)
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(m.count).astype(np.float32) * scale
    # Glorot-like scale per layer so that activations stay O(1)
    for l in range(m.L):
        fi = m.widths[l]
        o, n = m.w_off[l], m.widths[l] * m.widths[l + 1]
        p[o:o + n] *= 2.0 / math.sqrt(fi)
    m.p.copy_(torch.from_numpy(p))
    m.refresh_bf16()
    return m


def _ws_layers(m, ws, B):
    """(z_l, h_l) host arrays of the forward workspace, l = 1 .. L-1."""
    out, o = [], 0
    w = ws.cpu().numpy().astype(np.float64)
    for l in range(1, m.L):
        n = m.widths[l]
        z = w[o:o + B * n].reshape(B, n)
        h = w[o + B * n:o + 2 * B * n].reshape(B, n)
        out.append((z, h))
        o += 2 * B * n
    return out


SHAPES = [((8, 256, 256, 256, 256, 1), 4096 + 17), ((8, 256, 256, 256, 256, 1), 1),
          ((8, 16, 48, 1), 300), ((6, 32, 1), 127), ((8, 128, 64, 1), 128)]


@pytest.mark.parametrize("widths,B", SHAPES)
def test_layerwise_parity(mods, widths, B):
    _, surrogate = mods
    m = _mlp(surrogate, widths, 100 + B)
    rng = np.random.default_rng(B)
    x = rng.uniform(-1, 1, size=(B, widths[0])).astype(np.float32)
    y = m.forward(torch.from_numpy(x).cuda(), keep=True)
    torch.cuda.synchronize()
    W, b = m.weights()
    layers = _ws_layers(m, m._ws["ws"], B)
    h_in = ref.bf16_pair(x)
    for l, (zg, hg) in enumerate(layers):
        zr = h_in @ W[l].T + b[l]
        mag = np.abs(h_in) @ np.abs(W[l]).T + np.abs(b[l])
        K = W[l].shape[1]
        assert np.all(np.abs(zg - zr) <= 2 * K * 2.0 ** -24 * mag + 1e-30), (l, np.max(np.abs(zg - zr) / mag))
        # hidden activations are bfloat16 values: the rounded GELU of z
        hb = hg.astype(np.float32).view(np.uint32)
        assert np.all(hb & 0xFFFF == 0)
        g = ref.gelu(zg)
        assert np.all(np.abs(hg - g) <= 2.0 ** -8 * np.abs(g) + 2e-7 * (1.0 + np.abs(zg))), l
        h_in = hg
    yr = h_in @ W[-1][0] + b[-1][0]
    mag = np.abs(h_in) @ np.abs(W[-1][0]) + abs(b[-1][0])
    K = W[-1].shape[1]
    assert np.all(np.abs(y.cpu().numpy() - yr) <= 2 * K * 2.0 ** -24 * mag + 1e-30)


@pytest.mark.parametrize("widths,B", SHAPES[:3])
def test_end_to_end_against_the_bf16_reference(mods, widths, B):
    _, surrogate = mods
    m = _mlp(surrogate, widths, 200 + B)
    rng = np.random.default_rng(7 + B)
    x = rng.uniform(-1, 1, size=(B, widths[0])).astype(np.float32)
    y = m.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    W, b = m.weights()
    yr, _, _ = ref.forward(W, b, x, act_bf16=True)
    scale = 1.0 + np.max(np.abs(yr))
    assert np.max(np.abs(y - yr)) <= 3e-3 * scale
    # and the float32-activation network differs by the bfloat16 rounding itself
    y32, _, _ = ref.forward(W, b, x.astype(np.float64))
    assert np.max(np.abs(y - y32)) <= 3e-2 * scale


def test_inference_and_training_forward_agree(mods):
    _, surrogate = mods
    m = _mlp(surrogate, (8, 256, 256, 256, 256, 1), 5)
    x = torch.rand(5000, 8, device="cuda") * 2 - 1
    a = m.forward(x, keep=True)
    b = m.forward(x)
    assert torch.equal(a, b)


def test_gradients_from_the_tensor_core_forward(mods):
    # the backward pass differentiates the network as evaluated: the oracle's
    # chain rule fed with the GPU's own pre-activations and activations
    _, surrogate = mods
    widths = (8, 256, 256, 1)
    B = 2048
    m = _mlp(surrogate, widths, 9)
    rng = np.random.default_rng(10)
    x = rng.uniform(-1, 1, size=(B, 8)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    y, _ = m.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    torch.cuda.synchronize()
    W, b = m.weights()
    layers = _ws_layers(m, m._ws["ws"], B)
    zs = [z for z, _ in layers] + [None]
    hs = [ref.bf16_pair(x)] + [h for _, h in layers]
    dy = 2.0 * (y.cpu().numpy().astype(np.float64) - t) / B
    dW, db = ref.backward_from(W, zs, hs, dy)
    g = m.g.cpu().numpy().astype(np.float64)
    for l in range(len(W)):
        gw = g[m.w_off[l]:m.w_off[l] + W[l].size].reshape(W[l].shape)
        gb = g[m.b_off[l]:m.b_off[l] + b[l].size]
        for got, want in ((gw, dW[l]), (gb, db[l])):
            assert np.max(np.abs(got - want)) <= 1e-4 * (np.max(np.abs(want)) + 1e-30), l


def test_shapes_outside_the_tensor_core_path_are_rejected(mods):
    sfft, surrogate = mods
    with pytest.raises(ValueError):
        surrogate.MLP((8, 40, 1), tensor_cores=True)
    # through the C ABI: a 40-wide hidden layer in tensor-core mode
    m = surrogate.MLP((8, 40, 1), tensor_cores=False)
    m.net.mode = sfft.MLP_TENSOR_CORES
    x = torch.zeros(4, 8, device="cuda")
    y = torch.empty(4, device="cuda")
    sc = torch.empty(4 * 40 * 2, device="cuda")
    s = m.lib.sfft_mlp_forward(ctypes.byref(m.net), ctypes.c_void_p(x.data_ptr()), 4,
                               ctypes.c_void_p(y.data_ptr()), None, ctypes.c_void_p(sc.data_ptr()), None)
    assert s == sfft.SFFT_EINVAL


def test_no_tensor_core_wait_expired(mods):
    sfft, _ = mods
    assert sfft.load_library().sfft_mlp_tc_timeouts() == 0
