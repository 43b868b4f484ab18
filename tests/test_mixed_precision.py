"""Mixed precision (sfft_set_precision(SFFT_PRECISION_MIXED)): the zip-up's
MPO contraction in complex FP32 on the tensor cores, the QR/SVD steps in
FP64. Per-instance price error against the CPU oracle's FP64 discrete sum and
against the FP64 path, at the mixed configuration's tolerance 1e-7 with its
acceptance of 1e-6 S0 per instance.

The FP32 contraction (tf32 hi + lo operands, FP32 accumulation) leaves each
panel entry within a few FP32 roundings of its FP64 value, relative to the
sum of the magnitudes of its terms; the rounding sweep at tolerance 1e-7
dominates that, so the 1e-6 S0 acceptance (the configured target) holds with
margin. The mixed prices must also differ from the FP64 path's, which shows
that the contraction did not run in FP64.
"""
import math

import numpy as np
import pytest

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ACCEPT = 1e-6  # times S0, per instance


@pytest.fixture(scope="module")
def pricers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    fp64 = sfft.Pricer(0)
    mixed = sfft.Pricer(0)
    mixed.set_precision(True)
    yield fp64, mixed
    fp64.close()
    mixed.close()


def _errors(probs, strikes, prices, seed, sample=8, J=None):
    """Per-instance maximum |GPU - oracle| / S0 over sampled strikes."""
    c = prices.cpu().numpy()
    rng = np.random.default_rng(seed)
    out, off = [], 0
    for p, (lb, st, q) in zip(probs, strikes):
        u = wl.strike_set(lb, st, q)
        pick = np.unique(np.concatenate([[0, q - 1, q // 2], rng.integers(0, q, sample)]))
        ref, _ = cm.prices(p, u[pick], route="sparse", J=J)
        out.append(float(np.max(np.abs(c[off + pick] - ref))) / p.S0)
        off += q
    return np.array(out)


def test_config4_instances_against_the_oracle_and_the_fp64_path(pricers):
    fp64, mixed = pricers
    probs = wl.config3_batch(60, n_lo=30, n_hi=30, tol=1e-7)
    strikes = [cm.strike_window(p) for p in probs]
    mixed.profile(True)
    mixed.profile_read(reset=True)
    cm_, km, sm, _ = mixed.price_batch(probs, strikes, raise_on_error=False)
    prof = mixed.profile_read(reset=True)
    mixed.profile(False)
    c64, k64, s64, _ = fp64.price_batch(probs, strikes, raise_on_error=False)
    assert list(sm) == list(s64)
    ok = [i for i, s in enumerate(sm) if s == 0]
    assert len(ok) >= 55
    # the contraction ran on the tensor cores: sites were counted, and the
    # prices differ from the FP64 path's in their last digits. The sites
    # above a TT-SVD block (delta cores) come from the MPO's cached prefix,
    # which is the same for every instance and computed once in FP64; each
    # instance contracts its block's sites (support 2^6..2^14) on the tensor
    # cores
    assert prof["zipup"]["evals"] >= 5 * len(ok)
    a, b = cm_.cpu().numpy(), c64.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([q for _, _, q in strikes])])
    dev = np.array([np.max(np.abs(a[offs[i]:offs[i + 1]] - b[offs[i]:offs[i + 1]])) / probs[i].S0 for i in ok])
    assert np.max(dev) > 1e-13
    # every strike of every instance within the acceptance of the FP64 path
    assert np.max(dev) <= ACCEPT, np.max(dev)
    assert torch.equal(km, k64)
    # and sampled strikes of every instance whose direct sum runs over at most
    # 2^20 points within the acceptance of the oracle
    sel = [i for i in ok if cm.support_limit(probs[i]) <= (1 << 20)]
    assert len(sel) >= 30
    e = _errors([probs[i] for i in sel], [strikes[i] for i in sel],
                torch.cat([cm_[offs[i]:offs[i + 1]] for i in sel]), seed=40)
    assert np.all(e <= ACCEPT), (np.max(e), np.argmax(e))


@pytest.mark.parametrize("n", [16, 20, 24])
def test_all_models_small_n(pricers, n):
    _, mixed = pricers
    probs = [wl.config2_heston(n, tol=1e-7), wl.config1_gbm().replace(n=n, tol=1e-7)]
    probs += wl.config3_batch(9, seed=41 + n, n_lo=n, n_hi=n, tol=1e-7)
    strikes = [cm.strike_window(p) for p in probs]
    c, _, st, _ = mixed.price_batch(probs, strikes, raise_on_error=False)
    assert all(s == 0 for s in st), list(st)
    e = _errors(probs, strikes, c, seed=n, J=1 << n)
    assert np.all(e <= ACCEPT), e


def test_mixed_precision_in_a_captured_batch(pricers):
    from paper_2607_28435_b300 import sfft
    _, mixed = pricers
    probs = wl.config3_batch(12, seed=44, n_lo=30, n_hi=30, tol=1e-7)
    strikes = [cm.strike_window(p) for p in probs]
    c, k, st, _ = mixed.price_batch(probs, strikes, raise_on_error=False)
    g = sfft.Graph(mixed, probs, strikes)
    try:
        g.launch()
        gst, _ = g.status()
        assert gst == list(st)
        assert np.array_equal(g.prices.cpu().numpy(), c.cpu().numpy())
    finally:
        g.close()


def test_precision_mode_is_validated(pricers):
    from paper_2607_28435_b300 import sfft
    fp64, _ = pricers
    assert fp64.lib.sfft_set_precision(fp64.h, 7) == sfft.SFFT_EINVAL
