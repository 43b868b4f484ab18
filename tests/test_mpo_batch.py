"""The Q_n MPOs (Sec. 3.2) a pricing call needs are built together: one
interpolation launch per MPO, then one rounding launch with a CTA per MPO.
Each MPO's rounding runs on one CTA either way, so the batched build gives
the same cores, bit for bit, as building each MPO on its own; and the
priced batch agrees with the oracle whichever way its MPOs were built."""
import numpy as np
import pytest
import torch

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

pytestmark = pytest.mark.gpu

NS = (10, 13, 17, 22)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    return sfft


def _batch():
    return [wl.paper_grid_bs(n) for n in NS]


def test_batched_build_equals_one_at_a_time(lib):
    probs = _batch()
    tol = probs[0].tol
    # context 1: every MPO built by the batched path of one pricing call
    p1 = lib.Pricer(0)
    try:
        c1, _, st, _ = p1.price_batch(probs, [cm.strike_window(p, qmax=64) for p in probs])
        assert st == [0] * len(probs)
        batched = {n: p1.mpo(n, tol) for n in NS}
    finally:
        p1.close()
    # context 2: each MPO built on its own, in a different order
    p2 = lib.Pricer(0)
    try:
        single = {n: p2.mpo(n, tol) for n in reversed(NS)}
        c2, _, st2, _ = p2.price_batch(probs, [cm.strike_window(p, qmax=64) for p in probs])
        assert st2 == [0] * len(probs)
    finally:
        p2.close()
    for n in NS:
        a, b = batched[n], single[n]
        assert len(a) == len(b) == n
        for ga, gb in zip(a, b):
            assert ga.shape == gb.shape
            assert np.array_equal(ga, gb), n
    assert np.array_equal(c1.cpu().numpy(), c2.cpu().numpy())


def test_batched_build_prices_match_oracle(lib):
    probs = _batch()
    strikes = [cm.strike_window(p, qmax=64) for p in probs]
    p = lib.Pricer(0)
    try:
        c, lk, st, _ = p.price_batch(probs, strikes)
        assert st == [0] * len(probs)
        c = c.cpu().numpy()
        off = 0
        for prob, s in zip(probs, strikes):
            u = wl.strike_set(*s)
            ref, _ = cm.prices(prob, u, route="fft")
            got = c[off:off + s[2]]
            off += s[2]
            assert np.max(np.abs(got - ref)) <= 1e-8 * prob.S0, prob.n
    finally:
        p.close()
