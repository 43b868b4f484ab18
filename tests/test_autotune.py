"""Tuning of the first-tier carves (sfft_autotune, include/sfft.h): the tuned
configuration is cached under the batch's signature, used by later calls,
exported and imported as text so that a given cache fixes the choice without
re-timing, and prices as the defaults do (the carves change only how the
work is split, so the prices agree with the oracle's FP64 sum to 1e-8 S0)."""
import numpy as np
import pytest

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfft_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    return sfft


def test_tune_cache_round_trip_and_prices(sfft_mod):
    sfft = sfft_mod
    probs = wl.config3_batch(384, seed=77)
    strikes = [cm.strike_window(p) for p in probs]
    a = sfft.Pricer(0)
    b = sfft.Pricer(0)
    try:
        cfg0, found0 = a.tune_lookup(probs)
        assert not found0 and cfg0 == dict(build_p=32, round_r=24, zip_ctas=0)
        c_def, _, st_def, _ = a.price_batch(probs, strikes, raise_on_error=False)
        c_def = c_def.cpu().numpy()
        chosen, ms_c, ms_d = a.autotune(probs, strikes, reps=1)
        assert ms_c <= ms_d
        # the default and the five coordinate-descent candidates were timed
        trials = a.tune_trials()
        assert len(trials) == 6 and trials[0] == (cfg0, ms_d)
        assert min(m for _, m in trials) == ms_c
        cfg, found = a.tune_lookup(probs)
        assert found and cfg == chosen
        # another draw of the same workload shares the signature
        assert a.tune_lookup(wl.config3_batch(384, seed=78))[1]
        text = a.tune_export()
        assert text.count("\n") == 1
        # a fresh context with the imported cache makes the same choice, untimed
        b.tune_import(text)
        assert b.tune_lookup(probs) == (chosen, True)
        assert b.tune_export() == text
        c_t, _, st_t, _ = b.price_batch(probs, strikes, raise_on_error=False)
        assert list(st_t) == list(st_def)
        c_t = c_t.cpu().numpy()
        ok = np.repeat(np.array(list(st_t)) == 0, [q for _, _, q in strikes])
        assert np.max(np.abs(c_t[ok] - c_def[ok])) <= 1e-9 * 100.0
        # and sampled strikes against the oracle
        rng = np.random.default_rng(3)
        off = 0
        for p, (lb, sd, q), s in zip(probs[:40], strikes[:40], list(st_t)[:40]):
            if s == 0 and cm.support_limit(p) <= (1 << 20):
                u = wl.strike_set(lb, sd, q)
                pick = np.unique(np.concatenate([[0, q - 1], rng.integers(0, q, 4)]))
                ref, _ = cm.prices(p, u[pick])
                assert np.max(np.abs(c_t[off + pick] - ref)) <= 1e-8 * p.S0
            off += q
    finally:
        a.close()
        b.close()


def test_tune_import_rejects_malformed_text(sfft_mod):
    sfft = sfft_mod
    p = sfft.Pricer(0)
    try:
        for bad in ("no numbers here\n", "sm103 x148|count=1 33 24 0\n", "k 32 24\n"):
            with pytest.raises(sfft.SfftError) as ei:
                p.tune_import(bad)
            assert ei.value.status == sfft.SFFT_EINVAL
        assert p.tune_export() == ""
    finally:
        p.close()


def test_tuning_is_refused_under_the_tier1_hook(sfft_mod, monkeypatch):
    sfft = sfft_mod
    monkeypatch.setenv("SFFT_TIER1", "round=8")
    p = sfft.Pricer(0)
    try:
        probs = wl.config3_batch(8, seed=79)
        with pytest.raises(sfft.SfftError) as ei:
            p.autotune(probs, [cm.strike_window(q) for q in probs])
        assert ei.value.status == sfft.SFFT_EINVAL
    finally:
        p.close()
