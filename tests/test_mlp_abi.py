"""The surrogate's C ABI (include/sfft_mlp.h) without a GPU: the workspace
size formula, and the argument checks that reject a call before any device
work is enqueued."""
import ctypes

import pytest

from paper_2607_28435_b300 import build, sfft

c_void_p = ctypes.c_void_p


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sfft.load_library()


def _net(widths, ptrs=True):
    n = sfft.SfftMlp()
    n.n_layers = len(widths) - 1
    for i, w in enumerate(widths):
        n.width[i] = w
    for l in range(len(widths) - 1):
        # placeholders: these calls are rejected or need no device access
        n.w[l] = 0x1000 if ptrs else None
        n.b[l] = 0x2000 if ptrs else None
    return n


def test_workspace_floats(lib):
    # z_l and h_l of every hidden layer, batch rows each
    for widths, batch in (((8, 256, 256, 1), 10), ((8, 40, 70, 33, 1), 37), ((3, 1), 5)):
        want = sum(2 * batch * w for w in widths[1:-1])
        assert lib.sfft_mlp_workspace_floats(ctypes.byref(_net(widths)), batch) == want


@pytest.mark.parametrize("widths", [(8,), (8, 256, 2), (8, 2000, 1), (8, 0, 1),
                                    (8, 4, 4, 4, 4, 4, 4, 4, 4, 1)])
def test_bad_networks_are_rejected(lib, widths):
    n = _net(widths) if len(widths) <= sfft.MLP_MAX_LAYERS + 1 else None
    if n is None:
        n = _net(widths[:sfft.MLP_MAX_LAYERS + 1])
        n.n_layers = len(widths) - 1
    assert lib.sfft_mlp_workspace_floats(ctypes.byref(n), 4) == -1
    assert lib.sfft_mlp_forward(ctypes.byref(n), c_void_p(0x3000), 4, c_void_p(0x4000), c_void_p(0x5000),
                                None, None) == sfft.SFFT_EINVAL


def test_missing_pointers_are_rejected(lib):
    n = _net((8, 16, 1), ptrs=False)
    assert lib.sfft_mlp_forward(ctypes.byref(n), c_void_p(0x3000), 4, c_void_p(0x4000), c_void_p(0x5000),
                                None, None) == sfft.SFFT_EINVAL
    good = _net((8, 16, 1))
    # neither a workspace nor inference scratch for a network with a hidden layer
    assert lib.sfft_mlp_forward(ctypes.byref(good), c_void_p(0x3000), 4, c_void_p(0x4000), None, None,
                                None) == sfft.SFFT_EINVAL
    # more batch rows than the row tiles of one grid can address
    assert lib.sfft_mlp_forward(ctypes.byref(good), c_void_p(0x3000), 65536 * 64, c_void_p(0x4000),
                                c_void_p(0x5000), None, None) == sfft.SFFT_EINVAL
    gw = (c_void_p * 2)(None, None)
    assert lib.sfft_mlp_backward(ctypes.byref(good), c_void_p(0x3000), 4, c_void_p(0x5000), c_void_p(0x6000),
                                 gw, gw, c_void_p(0x7000), None) == sfft.SFFT_EINVAL


def test_other_entry_points_check_arguments(lib):
    assert lib.sfft_mlp_normalize(None, -1, 8, None, None, None, None, None) == sfft.SFFT_EINVAL
    assert lib.sfft_mlp_normalize(None, 4, 0, None, None, None, None, None) == sfft.SFFT_EINVAL
    assert lib.sfft_mlp_normalize(None, 0, 8, None, None, None, None, None) == sfft.SFFT_OK
    assert lib.sfft_mlp_mse_grad(None, None, 3, None, None, None) == sfft.SFFT_EINVAL
    assert lib.sfft_mlp_mse_grad(None, None, 0, None, None, None) == sfft.SFFT_OK
    assert lib.sfft_mlp_adam(-1, None, None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 1, None) == sfft.SFFT_EINVAL
    assert lib.sfft_mlp_adam(4, None, None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 1, None) == sfft.SFFT_EINVAL
    assert lib.sfft_mlp_adam(4, c_void_p(0x10), None, c_void_p(0x20), c_void_p(0x30), c_void_p(0x40), 1e-3,
                             0.9, 0.999, 1e-8, 0, None) == sfft.SFFT_EINVAL
    assert lib.sfft_mlp_adam(0, None, None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 1, None) == sfft.SFFT_OK
