"""QFT route by statevector emulation (Sec. 3, QFT-based option pricing), on
the GPU through the C ABI (sfft_qft_price_batch), against the oracle's
exact-probability readout (Eq. qft_observable_price) and the paper's printed
statevector errors (Sec. 4.2)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import carr_madan as cm
from oracle import closed_forms as cfm
from paper_2607_28435_b300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pricer():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    p = sfft.Pricer(0)
    yield p
    p.close()


def _full(prob):
    g = cm.grid(prob)
    return (0, 1, g["M"])


def _bs(K):
    return cfm.bs_call(100.0, K, 0.05, 0.3, 0.5)


@pytest.mark.parametrize("n", [3, 6, 9, 12, 16, 20])
def test_matches_oracle_abs_readout(pricer, n):
    # the emulated circuit and the oracle's |y| readout of the same sum agree
    # to rounding inside the evaluation window K in [50, 150]
    p = wl.paper_grid_bs(n)
    s = _full(p) if n <= 16 else cm.strike_window(p, qmax=4096)
    c, lk, st, _ = pricer.qft_price_batch([p], [s])
    assert st == [0]
    c, lk = c.cpu().numpy(), lk.cpu().numpy()
    u = wl.strike_set(*s)
    y = cm.y_full(p, "fft")[u]
    ref = cm.prices_qft_readout(p, u, y)
    K = np.exp(lk)
    win = (K >= 50) & (K <= 150)
    assert np.all(np.isfinite(c))
    assert np.max(np.abs(c[win] - ref[win])) <= 1e-10 * p.S0, n


def test_printed_statevector_nrmse(pricer):
    # Sec. 4.2 prints the statevector NRMSE against Black-Scholes at n = 3..5,
    # where the discretisation error dominates
    rows = []
    with open(os.path.join(GOLDEN, "paper_nrmse.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    checked = 0
    for n, val, how in rows:
        if how != "abs":
            continue
        n, val = int(n), float(val)
        p = wl.paper_grid_bs(n)
        c, lk, st, _ = pricer.qft_price_batch([p], [_full(p)])
        assert st == [0]
        e, cnt = cm.nrmse(p, c.cpu().numpy(), lk.cpu().numpy(), _bs)
        assert cnt > 0
        assert abs(e - val) <= 0.5e-2 * val + 0.005 * 10 ** math.floor(math.log10(val)), (n, e, val)
        checked += 1
    assert checked == 3


@pytest.mark.parametrize("n", [8, 14])
def test_probabilities_sum_to_one(pricer, n):
    # unitarity of the emulated circuit: with all M outcomes requested,
    # sum_l p_l = 1, i.e. sum_l (C_l / (S0 f_l))^2 = ||x||^2
    p = wl.paper_grid_bs(n)
    s = _full(p)
    c, _, st, _ = pricer.qft_price_batch([p], [s])
    assert st == [0]
    u = wl.strike_set(*s)
    scale, _ = cm.price_scale(p, u)
    amp = c.cpu().numpy() / (p.S0 * scale)
    x = cm.integrand(p, np.arange(1 << n))
    assert abs(np.sum(amp ** 2) / np.vdot(x, x).real - 1.0) <= 1e-12


def test_heston_agrees_with_real_part_on_symmetric_grid(pricer):
    # on the symmetric grid the sum is real up to its one unpaired term, so
    # the QFT route's |y| readout (the positive-phase assumption) matches the
    # dense route's real part to the price tolerance
    p = wl.Problem(wl.HESTON, wl.HESTON_CFG2, S0=100.0, r=0.025, T=1.0, alpha=1.5, eta=0.0,
                   n=16, quad=wl.RECT_SYM)
    s = cm.strike_window(p)
    cq, _, st1, _ = pricer.qft_price_batch([p], [s])
    cd, _, st2, _ = pricer.dense_price_batch([p], [s])
    assert st1 == [0] and st2 == [0]
    assert np.max(np.abs(cq.cpu().numpy() - cd.cpu().numpy())) <= 1e-8 * p.S0


def test_rejects_beyond_dense_limit_and_one_sided_grid(pricer):
    from paper_2607_28435_b300 import sfft
    p = wl.paper_grid_bs(33)
    _, _, st, _ = pricer.qft_price_batch([p], [cm.strike_window(p, qmax=16)], raise_on_error=False)
    assert st == [sfft.SFFT_EINVAL]
    # the Simpson grid's sum is not real: |y| would not be a price
    q = wl.config2_heston(16)
    c, _, st, _ = pricer.qft_price_batch([q], [cm.strike_window(q, qmax=16)], raise_on_error=False)
    assert st == [sfft.SFFT_EINVAL]
    assert np.all(np.isnan(c.cpu().numpy()))
