"""The zip-up's delta prefix (Sec. 3.2's MPO x TT contraction over the sites
above a TT-SVD block, whose integrand cores are the rank-one delta_{lam,0}).
That part of the zip-up depends on the MPO alone, so it is computed once per
cached MPO and copied into each instance's zip-up, which then starts at the
block's first site. The arithmetic is the same as running the zip-up from
site 0, so the prices and ranks must agree bit for bit with a context whose
SFFT_ZPRE=0 hook turns the prefix off, on a batch with TT-SVD and cross-built
instances, blocks of every size up to n, and several MPOs. The prices are
also checked against the oracle's FP64 discrete sum (1e-8 S0).
"""
import os

import numpy as np
import pytest

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pricers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    on = sfft.Pricer(0)
    old = os.environ.get("SFFT_ZPRE")
    os.environ["SFFT_ZPRE"] = "0"
    try:
        off = sfft.Pricer(0)
    finally:
        if old is None:
            del os.environ["SFFT_ZPRE"]
        else:
            os.environ["SFFT_ZPRE"] = old
    return sfft, on, off


def _batch():
    # the bench batch's first instances (n 16..34, all three models) plus a
    # block as wide as the grid (no delta site) and long delta prefixes (n = 40)
    probs = wl.config3_batch(96)
    g = wl.config1_gbm()
    probs += [g.replace(n=6), g.replace(n=8)]
    h = wl.config2_heston(40)
    probs += [h, h.replace(T=0.1), h.replace(n=24, T=3.0)]
    return probs


def test_prefix_bit_identical_and_priced():
    sfft, on, off = _pricers()
    try:
        probs = _batch()
        strikes = [sfft.strike_window(p) for p in probs]
        c1, k1, st1, info1 = on.price_batch(probs, strikes, raise_on_error=False)
        c0, k0, st0, info0 = off.price_batch(probs, strikes, raise_on_error=False)
        assert list(st1) == list(st0)
        assert [i["out_rank"] for i in info1] == [i["out_rank"] for i in info0]
        a1, a0 = c1.cpu().numpy(), c0.cpu().numpy()
        same = (a1 == a0) | (np.isnan(a1) & np.isnan(a0))
        assert same.all(), int((~same).sum())
        # and the prices themselves, at both ends of each window and its middle
        off_i = 0
        for p, (lb, stp, q), s in zip(probs, strikes, st1):
            if s == 0:
                u = wl.strike_set(lb, stp, q)
                pick = np.array(sorted({0, q // 2, q - 1}))
                ref, _ = cm.prices(p, u[pick], route="sparse")
                err = float(np.max(np.abs(a1[off_i + pick] - ref))) / p.S0
                assert err <= 1e-8, (p, err)
            off_i += q
    finally:
        on.close()
        off.close()


def test_prefix_cuts_zipup_work():
    # the profiler's algorithmic flops of the zip-up phase drop by the delta
    # sites' share; the other phases are unchanged
    sfft, on, off = _pricers()
    try:
        probs = wl.config3_batch(64)
        strikes = [sfft.strike_window(p) for p in probs]
        res = []
        for pr in (on, off):
            pr.price_batch(probs, strikes, raise_on_error=False)
            pr.profile(True)
            pr.profile_read()
            pr.price_batch(probs, strikes, raise_on_error=False)
            res.append(pr.profile_read())
            pr.profile(False)
        z1, z0 = res[0]["zipup"]["flops"], res[1]["zipup"]["flops"]
        assert 0 < z1 < 0.95 * z0, (z1, z0)
        assert res[0]["round"]["flops"] == res[1]["round"]["flops"]
    finally:
        on.close()
        off.close()
