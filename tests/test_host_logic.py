"""Host-side logic of the bench and the surrogate that needs no GPU: the
workload selection, the CPU-oracle sample's pieces, and the surrogate's
(T, k) trust cells."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import carr_madan as cm  # noqa: E402
from paper_2607_28435_b300 import workloads as wl  # noqa: E402


def _args(**kw):
    a = argparse.Namespace(count=64, n=None, tol=1e-12)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_default_and_fixed_n_workloads():
    a = _args()
    probs = bench.batch_problems(a)
    assert len(probs) == 64
    assert all(16 <= p.n <= 34 and p.tol == 1e-12 for p in probs)
    assert bench.workload_name(a) == "batched TT-SFFT, 64 instances (Heston/Merton/VG), n 16..34"
    # the default batch is the mixed batch itself
    ref = wl.config3_batch(64)
    assert [(p.model, p.p, p.T, p.n) for p in probs] == [(p.model, p.p, p.T, p.n) for p in ref]
    b = _args(n=30, tol=1e-7)
    probs = bench.batch_problems(b)
    assert all(p.n == 30 and p.tol == 1e-7 for p in probs)
    assert bench.workload_name(b).endswith("n 30, tol 1e-07")


def test_oracle_pieces_are_bounded_and_skip_wide_supports():
    probs = wl.config3_batch(256)
    strikes = [cm.strike_window(p) for p in probs]
    skipped = [0]
    seen = set()
    for i, (p, (lb, st, q)) in bench._oracle_pieces(probs, strikes, skipped, seed=1):
        m = cm.support_limit(p)
        assert m <= (1 << 20)
        assert q == min(strikes[i][2], max(32, (1 << 24) // m))
        assert lb == strikes[i][0] and st == strikes[i][1]
        assert i not in seen
        seen.add(i)
    wide = sum(cm.support_limit(p) > (1 << 20) for p in probs)
    assert skipped[0] == wide
    assert len(seen) + wide == len(probs)


def test_trust_cells_cover_the_box():
    from paper_2607_28435_b300.surrogate import Surrogate
    lo, hi = wl.SURROGATE_LO, wl.SURROGATE_HI
    raw = np.tile(np.array(lo, dtype=np.float64), (5, 1))
    raw[1, 6], raw[1, 7] = hi[6], hi[7]                      # the far corner
    raw[2, 6] = lo[6] + 0.5 * (hi[6] - lo[6])                 # the middle of T
    raw[3, 6], raw[3, 7] = lo[6] - 1.0, hi[7] + 1.0           # outside: clipped
    raw[4, 7] = lo[7] + (hi[7] - lo[7]) * 5.5 / 12            # inside k cell 5
    iT, ik = Surrogate.cells(raw, lo, hi, (6, 12))
    assert list(iT) == [0, 5, 3, 0, 0]
    assert list(ik) == [0, 11, 0, 11, 5]


def test_tuning_signature_buckets_batches_of_one_workload():
    # the tuning cache's batch signature (host only): the same workload drawn
    # with another seed shares it; another grid exponent, tolerance or size
    # does not
    from paper_2607_28435_b300 import sfft
    a = wl.config3_batch(4096)
    b = wl.config3_batch(4096, seed=wl.CONFIG3_SEED + 1)
    k = sfft.tune_key(a)
    assert k == sfft.tune_key(a) == sfft.tune_key(b)
    assert k != sfft.tune_key(wl.config3_batch(4096, n_lo=30, n_hi=30))
    assert k != sfft.tune_key(wl.config3_batch(4096, tol=1e-7))
    assert k != sfft.tune_key(a[:256])
    assert "tol=-12" in k and "count=13" in k
