"""Captured batches (sfft_graph_*): a replayed CUDA graph prices exactly what
sfft_price_batch prices, before and after a parameter update, and keeps
working after the calling context has priced other, larger batches."""
import numpy as np
import pytest
import torch

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pricer():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    p = sfft.Pricer(0)
    yield p
    p.close()


def _batch(count, seed):
    probs = wl.config3_batch(count, seed=seed)
    return probs, [cm.strike_window(p) for p in probs]


def _prices(pricer, probs, strikes, with_status=False):
    c, k, st, _ = pricer.price_batch(probs, strikes, raise_on_error=False)
    if with_status:
        return c.cpu().numpy(), k.cpu().numpy(), list(st)
    assert all(s == 0 for s in st)
    return c.cpu().numpy(), k.cpu().numpy()


def test_replays_match_price_batch(pricer):
    from paper_2607_28435_b300 import sfft
    probs, strikes = _batch(48, 11)
    ref_c, ref_k = _prices(pricer, probs, strikes)
    g = sfft.Graph(pricer, probs, strikes)
    try:
        for _ in range(2):
            g.prices.fill_(np.nan)
            g.launch()
            st, info = g.status(raise_on_error=True)
            assert st == [0] * len(probs)
            assert np.array_equal(g.prices.cpu().numpy(), ref_c)
            assert np.array_equal(g.log_strikes.cpu().numpy(), ref_k)
            assert max(i["out_rank"] for i in info) > 0
    finally:
        g.close()


def test_update_reprices_and_survives_other_batches(pricer):
    from paper_2607_28435_b300 import sfft
    probs, strikes = _batch(32, 12)
    g = sfft.Graph(pricer, probs, strikes)
    try:
        # new market data, same shape
        upd = [p.replace(S0=p.S0 * 1.1, r=p.r + 0.01, T=p.T * 0.9) for p in probs]
        g.update(upd)
        # the calling context prices a larger, different batch meanwhile
        big, big_s = _batch(256, 13)
        _prices(pricer, big, big_s, with_status=True)
        g.launch()
        st, _ = g.status()
        # the updated parameters may move an instance next to its moment
        # explosion (SFFT_EBOUNDS, prices still written): the replay and a
        # direct call agree on statuses and prices either way
        ref_c, ref_k, ref_st = _prices(pricer, upd, strikes, with_status=True)
        assert st == ref_st
        assert sum(s == 0 for s in st) >= len(st) - 2
        assert np.array_equal(g.prices.cpu().numpy(), ref_c)
        assert np.array_equal(g.log_strikes.cpu().numpy(), ref_k)
    finally:
        g.close()


def test_update_rejects_shape_change(pricer):
    from paper_2607_28435_b300 import sfft
    probs, strikes = _batch(4, 14)
    g = sfft.Graph(pricer, probs, strikes)
    try:
        bad = [probs[0].replace(n=probs[0].n + 1)] + list(probs[1:])
        with pytest.raises(sfft.SfftError):
            g.update(bad)
        g.launch()
        st, _ = g.status()
        assert st == [0] * len(probs)
    finally:
        g.close()


def test_create_refuses_failing_instance(pricer):
    from paper_2607_28435_b300 import sfft
    probs, strikes = _batch(2, 15)
    # an instance that cannot price (negative maturity)
    bad = probs[0].replace(T=-1.0)
    with pytest.raises(sfft.SfftError):
        sfft.Graph(pricer, probs + [bad], strikes + [strikes[0]])


def test_replays_match_the_oracle(pricer):
    # replays before and after an update, checked against the CPU oracle's
    # FP64 discrete sum at sampled strikes (1e-8 S0), not only against a
    # direct call
    from paper_2607_28435_b300 import sfft
    probs, strikes = _batch(24, 16)
    g = sfft.Graph(pricer, probs, strikes)
    rng = np.random.default_rng(16)
    try:
        upd = [p.replace(S0=90.0, T=p.T * 0.8, r=0.03) for p in probs]
        for stmt in (probs, upd):
            if stmt is upd:
                g.update(upd)
            g.prices.fill_(np.nan)
            g.launch()
            st, _ = g.status()
            c = g.prices.cpu().numpy()
            k = g.log_strikes.cpu().numpy()
            off, checked = 0, 0
            for p, (lb, sd, q), s in zip(stmt, strikes, st):
                if s == 0 and cm.support_limit(p) <= (1 << 20):
                    u = wl.strike_set(lb, sd, q)
                    pick = np.unique(np.concatenate([[0, q - 1], rng.integers(0, q, 6)]))
                    ref, kref = cm.prices(p, u[pick], route="sparse")
                    assert np.max(np.abs(c[off + pick] - ref)) <= 1e-8 * p.S0, p
                    assert np.max(np.abs(k[off + pick] - kref)) < 1e-12
                    checked += 1
                off += q
            assert checked >= 16, checked
    finally:
        g.close()
