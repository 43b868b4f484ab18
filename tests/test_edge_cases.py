"""Edge cases of the pricing path against the CPU oracle (1e-8 S0): the
largest grid exponent the library takes (n = 48), a strike set at the
per-instance limit of 65,536 strikes (and one past it, rejected), the
smallest grids (n = 1..4) on both quadrature rules, and a ragged batch whose
instances have 0, 1, a few or thousands of strikes at assorted strides."""
import math

import numpy as np
import pytest

from oracle import carr_madan as cm
from oracle import cf
from paper_2607_28435_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRICE_TOL = 1e-8  # times S0


@pytest.fixture(scope="module")
def pricer():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    p = sfft.Pricer(0)
    yield p
    p.close()


def _check(pricer, probs, strikes, picks=8, seed=0, route="sparse"):
    c, lk, st, _ = pricer.price_batch(probs, strikes, raise_on_error=False)
    assert list(st) == [0] * len(probs), list(st)
    c, lk = c.cpu().numpy(), lk.cpu().numpy()
    rng = np.random.default_rng(seed)
    off = 0
    for p, (lb, sd, q) in zip(probs, strikes):
        if q:
            u = wl.strike_set(lb, sd, q)
            pick = np.unique(np.concatenate([[0, q - 1, q // 2], rng.integers(0, q, picks)]))
            ref, kref = cm.prices(p, u[pick], route=route)
            assert np.max(np.abs(c[off + pick] - ref)) <= PRICE_TOL * p.S0, (p, q)
            assert np.max(np.abs(lk[off + pick] - kref)) < 1e-10
        off += q


def test_largest_grid_exponent(pricer):
    # n = SFFT_MAX_N = 48: 2.8e14 grid points held as a 48-site tensor train
    from paper_2607_28435_b300 import sfft
    probs = [wl.config2_heston(sfft.MAX_N),
             wl.Problem(cf.MERTON, (0.2, 0.8, -0.1, 0.15), S0=100.0, r=0.03, T=0.7, n=sfft.MAX_N)]
    _check(pricer, probs, [cm.strike_window(p) for p in probs], seed=48)
    bad = probs[0].replace(n=sfft.MAX_N + 1)
    with pytest.raises(sfft.SfftError):
        pricer.price_batch([bad], [(0, 1, 1)])


def test_strike_set_at_the_limit(pricer):
    from paper_2607_28435_b300 import sfft
    p = wl.config2_heston(22)
    lb, sd, q = cm.strike_window(p, qmax=sfft.MAX_STRIKES)
    assert q > sfft.MAX_STRIKES // 2
    _check(pricer, [p], [(lb, sd, q)], picks=24, seed=22)
    # exactly the limit, on a grid of 2^16 points: every grid strike
    g = wl.config1_gbm().replace(n=16)
    c, _, st, _ = pricer.price_batch([g], [(0, 1, sfft.MAX_STRIKES)], raise_on_error=False)
    assert list(st) in ([0], [sfft.SFFT_EBOUNDS])
    ref, kref = cm.prices(g, np.arange(1 << 16), route="fft")
    k = kref - math.log(g.S0)
    # the discrete sum's own rounding grows as e^{-alpha k} away from the money
    scale = g.S0 * np.maximum(1.0, np.exp(-g.alpha * k))
    assert np.all(np.abs(c.cpu().numpy() - ref) <= PRICE_TOL * scale)
    with pytest.raises(sfft.SfftError) as ei:
        pricer.price_batch([g], [(0, 1, sfft.MAX_STRIKES + 1)])
    assert ei.value.status == sfft.SFFT_EINVAL
    # a rejected strike count far over the limit: NaN prices of that length
    # (no host buffer of the limit's size is involved), the rest of the batch priced
    lb, sd, _ = cm.strike_window(g)
    for fn in (pricer.price_batch, pricer.dense_price_batch):
        c, _, st, _ = fn([g, g], [(0, 1, 1 << 19), (lb, sd, 4)], raise_on_error=False)
        assert list(st) == [sfft.SFFT_EINVAL, 0]
        c = c.cpu().numpy()
        assert np.all(np.isnan(c[:1 << 19])) and np.all(np.isfinite(c[1 << 19:]))


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_smallest_grids(pricer, n):
    # both quadrature rules; every grid point as a strike; the oracle's dense DFT
    probs = [wl.config1_gbm().replace(n=n), wl.paper_grid_bs(max(n, 2))]
    strikes = [(0, 1, 1 << p.n) for p in probs]
    c, _, st, _ = pricer.price_batch(probs, strikes, raise_on_error=False)
    c = c.cpu().numpy()
    off = 0
    for p, s, (_, _, q) in zip(probs, st, strikes):
        ref, _ = cm.prices(p, np.arange(q), route="direct")
        k = cm.log_moneyness(p, np.arange(q))
        scale = p.S0 * np.maximum(1.0, np.exp(-p.alpha * k))
        assert np.all(np.abs(c[off:off + q] - ref) <= PRICE_TOL * scale), (p.n, p.quad)
        off += q


def test_ragged_batch(pricer):
    # instances with 0, 1, 2, 3 and thousands of strikes, strides 1..2^t,
    # grid exponents 16..34, in one call
    rng = np.random.default_rng(5)
    probs = wl.config3_batch(36, seed=505)
    strikes = []
    for i, p in enumerate(probs):
        lb, sd, q = cm.strike_window(p)
        kind = i % 6
        if kind == 0:
            strikes.append((lb, sd, 0))
        elif kind in (1, 2, 3):
            strikes.append((lb + sd * int(rng.integers(0, q)), sd, 1) if kind == 1 else (lb, sd, kind))
        elif kind == 4:
            lb2 = -(-lb // (2 * sd)) * 2 * sd  # the first index aligned to the doubled stride
            strikes.append((lb2, 2 * sd, max((q - 1) // 2, 1)))
        else:
            strikes.append((lb, sd, q))
    sel = [i for i, p in enumerate(probs) if cm.support_limit(p) <= (1 << 20)]
    _check(pricer, [probs[i] for i in sel], [strikes[i] for i in sel], seed=6)
    # the whole batch in one call: statuses and the zero-strike instances
    c, _, st, _ = pricer.price_batch(probs, strikes, raise_on_error=False)
    assert all(s in (0, 8) for s in st)
    assert c.numel() == sum(q for _, _, q in strikes)
