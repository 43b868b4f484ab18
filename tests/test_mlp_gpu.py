"""The surrogate's CUDA kernels (include/sfft_mlp.h) against the FP64
reference of oracle/mlp.py, on the same bfloat16 weights: forward values,
gradients of every weight and bias (ragged tiles, and the split reduction
over large batches), one Adam step with its bfloat16 image, the input map;
then a small fit whose loss falls, queries answered by the network much
faster than by pricing each one, and the SFFT fallback outside the box."""
import math
import time

import numpy as np
import pytest
import torch

from oracle import mlp as ref
from paper_2607_28435_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft, surrogate
    build.build()
    return sfft, surrogate


def _random_mlp(surrogate, widths, seed, tensor_cores=False):
    # CUDA-core products (float32 activations) unless asked otherwise: the
    # tensor-core arithmetic has its own tests (test_mlp_tc.py)
    m = surrogate.MLP(widths, seed=seed, tensor_cores=tensor_cores)
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(m.count).astype(np.float32) * 0.4
    m.p.copy_(torch.from_numpy(p))
    m.refresh_bf16()
    return m


@pytest.mark.parametrize("widths,batch", [((8, 40, 70, 33, 1), 37), ((8, 40, 70, 33, 1), 130),
                                          ((8, 64, 64, 1), 2000), ((8, 256, 256, 1), 4096)])
def test_forward_and_gradients_match_oracle(mods, widths, batch):
    _, surrogate = mods
    m = _random_mlp(surrogate, widths, 11 + batch)
    rng = np.random.default_rng(batch)
    x = rng.uniform(-1, 1, size=(batch, widths[0])).astype(np.float32)
    t = rng.standard_normal(batch).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    y, loss = m.gradients(xd, td)
    torch.cuda.synchronize()
    W, b = m.weights()
    yr, _, _ = ref.forward(W, b, x.astype(np.float64))
    scale = 1.0 + np.max(np.abs(yr))
    assert np.max(np.abs(y.cpu().numpy() - yr)) <= 2e-5 * scale
    assert abs(float(loss.item()) - np.mean((yr - t) ** 2)) <= 1e-4 * (1.0 + np.mean((yr - t) ** 2))
    dW, db, _ = ref.backward(W, b, x.astype(np.float64), t.astype(np.float64))
    g = m.g.cpu().numpy().astype(np.float64)
    for l in range(len(W)):
        gw = g[m.w_off[l]:m.w_off[l] + W[l].size].reshape(W[l].shape)
        gb = g[m.b_off[l]:m.b_off[l] + b[l].size]
        for got, want in ((gw, dW[l]), (gb, db[l])):
            assert np.max(np.abs(got - want)) <= 1e-4 * (np.max(np.abs(want)) + 1e-30), (l, widths, batch)


def test_adam_step_and_bf16_image_match_oracle(mods):
    _, surrogate = mods
    m = _random_mlp(surrogate, (8, 16, 1), 5)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(m.count).astype(np.float32)
    p0 = m.p.cpu().numpy().astype(np.float64)
    m.g.copy_(torch.from_numpy(g))
    m.adam(1e-2)
    torch.cuda.synchronize()
    p_ref = p0.copy()
    mm, vv = np.zeros(m.count), np.zeros(m.count)
    ref.adam_step(p_ref, g.astype(np.float64), mm, vv, 1, 1e-2, 0.9, 0.999, 1e-8)
    p = m.p.cpu().numpy()
    assert np.max(np.abs(p - p_ref)) <= 1e-6
    # the bfloat16 image is the nearest bfloat16 of the float32 master copy
    want = ref.bf16_round(p)
    got = (m.p16.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


def test_normalize_and_box_flags(mods):
    _, surrogate = mods
    m = surrogate.MLP((8, 4, 1), seed=1, tensor_cores=False)
    lo, hi = np.array(wl.SURROGATE_LO), np.array(wl.SURROGATE_HI)
    rng = np.random.default_rng(7)
    raw = lo + (hi - lo) * rng.uniform(-0.2, 1.2, size=(257, 8))
    raw[0] = lo
    raw[1] = hi
    x, ib = m.normalize(torch.from_numpy(raw).cuda())
    want_x = 2.0 * (raw - lo) / (hi - lo) - 1.0
    assert np.max(np.abs(x.cpu().numpy() - want_x)) <= 1e-6
    want_in = np.all((raw >= lo) & (raw <= hi), axis=1)
    assert np.array_equal(ib.cpu().numpy().astype(bool), want_in)


def test_small_fit_and_serving(mods):
    sfft, surrogate = mods
    pricer = sfft.Pricer(0)
    try:
        # a narrow box around one parameter set: a small network fits it in seconds
        mid = [0.5 * (a + b) for a, b in zip(wl.SURROGATE_LO, wl.SURROGATE_HI)]
        lo = tuple(mid[:7]) + (-0.4,)
        hi = tuple(v * 1.05 if v > 0 else v * 0.95 for v in mid[:7]) + (0.4,)
        lo, hi = tuple(min(a, b) for a, b in zip(lo, hi)), tuple(max(a, b) for a, b in zip(lo, hi))
        sur, st = surrogate.train_surrogate(pricer, n_train_inst=64, n_test_inst=8, epochs=20, qmax=4096,
                                            widths=(8, 64, 64, 1), lo=lo, hi=hi, accept=1e-2)
        assert st["final_loss"] < 1e-3
        assert math.isfinite(st["heldout_max_abs_err"])
        # held-out queries: grid strikes of fresh instances inside the box
        test = wl.heston_surrogate_batch(4, 99, lo=lo, hi=hi)
        Xh, Yh = surrogate.sfft_dataset(pricer, test, kmin=lo[7], kmax=hi[7])
        Xh, Yh = Xh[:2048], Yh[:2048]
        # the fallback's grid mapping: rows that are grid strikes price as in the batch
        fp, fst = sur.sfft_prices(Xh[:16])
        assert np.allclose(fp, 100.0 * Yh[:16], rtol=0, atol=1e-8 * 100.0) and not fst.any()
        out, used, qst = sur.price(Xh)
        assert not qst.any()
        # the network answers only in trusted cells, within the acceptance
        # there; every other query is the SFFT price itself
        iT, ik = sur.cells(Xh, lo, hi, sur.trusted_cells.shape)
        assert np.array_equal(used, sur.trusted_cells[iT, ik])
        if used.any():
            assert np.max(np.abs(out[used] - 100.0 * Yh[used])) <= 1e-2 * 100.0
        assert np.allclose(out[~used], 100.0 * Yh[~used], rtol=0, atol=1e-8 * 100.0)
        # a chain (one parameter set, many strikes) shares one fallback instance
        # and prices as the per-query instances do
        chain = np.repeat(Xh[:1], 40, axis=0)
        chain[:, 7] = Xh[:40, 7] if np.all(Xh[:40, :7] == Xh[0, :7]) else np.linspace(lo[7], hi[7], 40)
        single = np.concatenate([sur.sfft_prices(chain[j:j + 1])[0] for j in range(0, 40, 13)])
        shared = sur.sfft_prices(chain)[0][::13]
        assert np.allclose(shared, single, rtol=0, atol=1e-8 * 100.0)
        # out of the box: answered by the SFFT pricer at the nearest grid strike
        far = Xh[:3].copy()
        far[:, 7] = 1.0  # log-moneyness outside [-0.4, 0.4]
        out_far, used_far, _ = sur.price(far)
        assert not used_far.any()
        assert np.allclose(out_far, sur.sfft_prices(far)[0], rtol=0, atol=1e-9 * 100.0)
        # throughput: the network against one SFFT instance per query
        B = 1 << 16
        rng = np.random.default_rng(8)
        q = np.asarray(lo) + (np.asarray(hi) - np.asarray(lo)) * rng.uniform(size=(B, 8))
        qd = torch.from_numpy(q).cuda()
        x, _ = sur.mlp.normalize(qd, lo, hi)
        sur.mlp.forward(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sur.mlp.forward(x)
        torch.cuda.synchronize()
        net_rate = B / (time.perf_counter() - t0)
        t0 = time.perf_counter()
        sur.sfft_prices(q[:512])
        sfft_rate = 512 / (time.perf_counter() - t0)
        assert net_rate > 20 * sfft_rate, (net_rate, sfft_rate)
    finally:
        pricer.close()


def test_fallback_statuses_reach_the_caller(mods):
    # a query next to a Heston moment explosion of order alpha + 1 (its
    # discrete sum leaves the no-arbitrage bounds, SFFT_EBOUNDS) and one whose
    # moment explodes before T (SFFT_EMOMENT, NaN price) come back flagged,
    # as does every query of a chain that shares such an instance; ordinary
    # queries come back 0
    sfft, surrogate = mods
    pricer = sfft.Pricer(0)
    try:
        net = surrogate.MLP((8, 16, 1), seed=2)
        sur = surrogate.Surrogate(pricer, net, np.full((6, 12), np.inf))  # trusts no cell
        bad = wl.heston_surrogate_batch(16384, 260728435)[8441]
        rows = [list(bad.p) + [bad.r, bad.T, k] for k in (-0.2, 0.0, 0.3)]
        rows.append(list(bad.p[:2]) + [0.99, 0.0, bad.p[4], 0.0, 2.99, 0.1])   # explodes before T
        rows.append(list(wl.HESTON_CFG2) + [0.025, 1.0, 0.1])                 # ordinary
        out, used, st = sur.price(np.array(rows))
        assert not used.any()
        assert list(st[:3]) == [sfft.SFFT_EBOUNDS] * 3, st
        assert st[3] == sfft.SFFT_EMOMENT and np.isnan(out[3])
        assert st[4] == 0 and np.isfinite(out[4])
    finally:
        pricer.close()


def test_surrogate_meets_the_acceptance_on_a_reduced_box(mods):
    # the learned part's acceptance, 1e-3 S0 in the maximum norm, on a reduced
    # Heston box (0.15 of every parameter range around the box centre,
    # |log-moneyness| <= 0.4): a fit of about 15 s on the tensor-core path;
    # trust is decided on the held-out set, the margin on the validation set,
    # and the figures asserted come from a third, independent set
    sfft, surrogate = mods
    pricer = sfft.Pricer(0)
    try:
        mid = [0.5 * (a + b) for a, b in zip(wl.SURROGATE_LO, wl.SURROGATE_HI)]
        span = [b - a for a, b in zip(wl.SURROGATE_LO, wl.SURROGATE_HI)]
        lo = tuple(m - 0.075 * s for m, s in zip(mid[:7], span[:7])) + (-0.4,)
        hi = tuple(m + 0.075 * s for m, s in zip(mid[:7], span[:7])) + (0.4,)
        t0 = time.perf_counter()
        sur, st = surrogate.train_surrogate(pricer, n_train_inst=4096, n_test_inst=512, epochs=300,
                                            widths=(8, 256, 256, 256, 1), lo=lo, hi=hi, qmax=256, cells=(4, 6),
                                            seed=11, lr=3e-3)
        assert time.perf_counter() - t0 < 90
        assert st["tensor_cores"]
        assert st["confirm_trusted_fraction"] >= 0.5, st
        assert st["confirm_max_abs_err_trusted"] <= 1e-3 * 100.0, st
        # served queries from fresh instances: network answers within the
        # acceptance, the rest priced by SFFT itself
        fresh = wl.heston_surrogate_batch(16, 12345, lo=lo, hi=hi)
        Xq, Yq = surrogate.sfft_dataset(pricer, fresh, qmax=64, kmin=lo[7], kmax=hi[7])
        out, used, qst = sur.price(Xq)
        assert not qst.any()
        if used.any():
            assert np.max(np.abs(out[used] - 100.0 * Yq[used])) <= 1e-3 * 100.0
        assert np.allclose(out[~used], 100.0 * Yq[~used], rtol=0, atol=1e-8 * 100.0)
    finally:
        pricer.close()
