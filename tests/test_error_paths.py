"""Failure paths and the second tier of the two-tier launches, through the C ABI.

Every failure here is made on the host (test hooks read by sfft_create from
the environment, see include/sfft.h): a narrowed first-tier limit, an
allocation that reports failure, a Jacobi sweep cap, a builder status
replaced by SFFT_ENOCONV. Nothing faults or stalls the device. Each test
checks the statuses, that failed instances carry NaN prices, that the rest of
the batch still prices to the oracle's FP64 discrete sum (1e-8 S0), and that
the context stays usable afterwards.
"""
import math

import numpy as np
import pytest

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRICE_TOL = 1e-8  # times S0


def _pricer():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    return sfft.Pricer(0)


def _check(prices, probs, strikes, status, ok_only=True, sample=8, seed=0, J=None):
    """Oracle check of sampled strikes of every status-0 instance; NaN prices
    for every other one. Returns the worst error over S0."""
    c = prices.cpu().numpy()
    rng = np.random.default_rng(seed)
    off, worst = 0, 0.0
    for p, (lb, st, q), s in zip(probs, strikes, status):
        u = wl.strike_set(lb, st, q)
        if s == 0:
            pick = np.unique(np.concatenate([[0, q - 1, q // 2], rng.integers(0, q, sample)]))
            ref, _ = cm.prices(p, u[pick], route="sparse", J=J)
            err = float(np.max(np.abs(c[off + pick] - ref))) / p.S0
            worst = max(worst, err)
            assert err <= PRICE_TOL, (p, err)
        elif ok_only:
            assert np.all(np.isnan(c[off:off + q])), (p, s)
        off += q
    return worst


def _mixed(count, seed, n_lo=16, n_hi=20):
    return wl.config3_batch(count, seed=seed, n_lo=n_lo, n_hi=n_hi)


def _heavy_vg(n, k=3):
    """Variance-Gamma draws with slowly decaying integrands (small T/nu): the
    cross builder takes them."""
    b = wl.config3_batch()
    return [q.replace(n=n) for q in b if q.model == wl.VG and q.T / q.p[1] < 0.6][:k]


# ------------------------------------------------------------- tier 2 -----
TIER1 = "build=8,round=6,cross=4,zipq=40,zipw=900"


def test_tier2_handoffs_match_oracle(monkeypatch):
    # narrowed first-tier limits: the TT-SVD builder hands on every instance
    # whose panels pass 8 columns (rank 4) part-way up the block, the zip-up
    # every instance with a panel of more than 40 columns part-way along the
    # chain, the rounding every output rank above 6; panels above 900 elements
    # are factored in global memory in tier 1 and by the streaming QR with an
    # explicit basis in tier 2. Tier 2 restarts each handed-on instance from
    # its unmodified inputs; prices must still match the oracle.
    monkeypatch.setenv("SFFT_TIER1", TIER1)
    pr = _pricer()
    try:
        probs = _mixed(30, 901) + [wl.config2_heston(24)]
        strikes = [cm.strike_window(p) for p in probs]
        prices, _, status, info = pr.price_batch(probs, strikes, raise_on_error=False)
        assert list(status) == [0] * len(probs), list(status)
        t2 = pr.tier2_counts()
        assert t2["build"] > 0 and t2["zipup"] > 0 and t2["round"] > 0, t2
        _check(prices, probs, strikes, status, seed=1)
        # the cross builder: ranks above 4 hand the instance on mid-sweep
        heavy = _heavy_vg(20)
        hs = [cm.strike_window(p) for p in heavy]
        prices, _, status, _ = pr.price_batch(heavy, hs, raise_on_error=False)
        assert list(status) == [0] * len(heavy), list(status)
        assert pr.tier2_counts()["cross"] > 0
        _check(prices, heavy, hs, status, seed=2, J=1 << 20)
    finally:
        pr.close()


def test_default_limits_keep_the_batch_in_tier1():
    # with the carves' own limits the mixed batch stays in tier 1 (its
    # second-tier launches have no work), which the hook test above is the
    # complement of
    pr = _pricer()
    try:
        probs = _mixed(64, 902, 16, 34)
        strikes = [cm.strike_window(p) for p in probs]
        pr.price_batch(probs, strikes, raise_on_error=False)
        t2 = pr.tier2_counts()
        assert t2 == dict(build=0, cross=0, zipup=0, round=0), t2
    finally:
        pr.close()


# --------------------------------------------------------------- ERANK ----
def test_erank_from_builder_and_rounding():
    from paper_2607_28435_b300 import sfft
    pr = _pricer()
    try:
        base = wl.config2_heston(20)
        good = wl.config1_gbm()
        strikes = [cm.strike_window(base), cm.strike_window(good)]
        _, _, st, info = pr.price_batch([base, good], strikes)
        a, b = info[0]["int_rank"], info[0]["out_rank"]
        assert 2 <= a < b, (a, b)
        # a cap below the integrand rank stops the builder
        probs = [base.replace(max_rank=a - 1), good]
        prices, _, status, _ = pr.price_batch(probs, strikes, raise_on_error=False)
        assert list(status) == [sfft.SFFT_ERANK, 0], list(status)
        _check(prices, probs, strikes, status, seed=3)
        # a cap between the two stops the output rounding
        probs = [base.replace(max_rank=a), good]
        prices, _, status, _ = pr.price_batch(probs, strikes, raise_on_error=False)
        assert list(status) == [sfft.SFFT_ERANK, 0], list(status)
        _check(prices, probs, strikes, status, seed=4)
        # the call reports the first failing status
        with pytest.raises(sfft.SfftError) as ei:
            pr.price_batch(probs, strikes)
        assert ei.value.status == sfft.SFFT_ERANK
    finally:
        pr.close()


# ------------------------------------------------------------- ENOCONV ----
def test_enoconv_from_jacobi_sweep_cap(monkeypatch):
    # one Jacobi sweep per SVD: the SVDs of the builder report non-convergence
    # on the device, the instances fail with SFFT_ENOCONV and NaN prices
    from paper_2607_28435_b300 import sfft
    monkeypatch.setenv("SFFT_FAULT", "jacobi:1")
    pr = _pricer()
    try:
        probs = [wl.config1_gbm(), wl.config2_heston(18)]
        strikes = [cm.strike_window(p) for p in probs]
        prices, _, status, _ = pr.price_batch(probs, strikes, raise_on_error=False)
        assert list(status) == [sfft.SFFT_ENOCONV] * 2, list(status)
        assert bool(torch.isnan(prices).all())
    finally:
        pr.close()
    # the cap belongs to that context's calls: a fresh context prices
    monkeypatch.delenv("SFFT_FAULT")
    pr = _pricer()
    try:
        prices, _, status, _ = pr.price_batch(probs, strikes, raise_on_error=False)
        assert list(status) == [0, 0]
        _check(prices, probs, strikes, status, seed=5)
    finally:
        pr.close()


def test_enoconv_of_one_instance_leaves_the_batch(monkeypatch):
    from paper_2607_28435_b300 import sfft
    monkeypatch.setenv("SFFT_FAULT", "enoconv:2")
    pr = _pricer()
    try:
        probs = _mixed(6, 903)
        strikes = [cm.strike_window(p) for p in probs]
        prices, _, status, _ = pr.price_batch(probs, strikes, raise_on_error=False)
        want = [0, 0, sfft.SFFT_ENOCONV, 0, 0, 0]
        assert list(status) == want, list(status)
        _check(prices, probs, strikes, status, seed=6)
    finally:
        pr.close()


# -------------------------------------------------------------- ENOMEM ----
def test_enomem_is_reported_and_the_context_recovers(monkeypatch):
    from paper_2607_28435_b300 import sfft
    monkeypatch.setenv("SFFT_FAULT", "enomem:zip_scratch:1")
    pr = _pricer()
    try:
        probs = _mixed(5, 904)
        strikes = [cm.strike_window(p) for p in probs]
        with pytest.raises(sfft.SfftError) as ei:
            pr.price_batch(probs, strikes)
        assert ei.value.status == sfft.SFFT_ENOMEM
        assert "zip_scratch" in str(ei.value)
        # the injected failure was one-shot: the same context prices next
        prices, _, status, _ = pr.price_batch(probs, strikes, raise_on_error=False)
        assert list(status) == [0] * len(probs)
        _check(prices, probs, strikes, status, seed=7)
    finally:
        pr.close()


def test_enomem_of_the_dense_buffer(monkeypatch):
    from paper_2607_28435_b300 import sfft
    monkeypatch.setenv("SFFT_FAULT", "enomem:dense_x")
    pr = _pricer()
    try:
        p = wl.config1_gbm()
        with pytest.raises(sfft.SfftError) as ei:
            pr.dense_price_batch([p], [cm.strike_window(p)])
        assert ei.value.status == sfft.SFFT_ENOMEM
        # the TT path needs no such buffer and still prices
        prices, _, status, _ = pr.price_batch([p], [cm.strike_window(p)])
        assert list(status) == [0]
        assert math.isfinite(float(prices[0]))
    finally:
        pr.close()
