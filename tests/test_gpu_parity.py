"""GPU parity: every step of the CUDA path, called through the C ABI, against
the CPU oracle on the same seeded inputs.

Tolerances: prices within 1e-8 * S0 of the oracle's FP64 discrete sum (the
FP64 target); intermediate tensors within a small multiple of the truncation
tolerance times the norm, which is what TT rounding guarantees.
"""
import math

import numpy as np
import pytest

from oracle import carr_madan as cm
from oracle import cf, closed_forms as cfm, tt
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


def bits_of(u, n):
    """Output-site physical indices of grid index u (site l carries bit l-1)."""
    return [(u >> s) & 1 for s in range(n)]


MODELS = {
    cf.GBM: (0.25,),
    cf.HESTON: wl.HESTON_CFG2,
    cf.MERTON: (0.2, 0.8, -0.1, 0.15),
    cf.VG: (0.2, 0.3, -0.14),
}


# ------------------------------------------------------------------ K1 ----
@pytest.mark.parametrize("model", list(MODELS))
@pytest.mark.parametrize("quad", [wl.SIMPSON_CM99, wl.RECT_SYM])
def test_integrand_samples(pricer, model, quad):
    rng = np.random.default_rng(100 + model + 10 * quad)
    for n in (6, 16, 30, 40):
        prob = wl.Problem(model, MODELS[model], S0=100.0, r=0.03, T=0.8, alpha=1.5,
                          eta=0.25 if quad == wl.SIMPSON_CM99 else 0.0, n=n, quad=quad)
        M = 1 << n
        j = np.unique(np.concatenate([np.arange(min(M, 64)), rng.integers(0, M, 200),
                                      [M - 1, M // 2, M // 2 - 1]])).astype(np.int64)
        got = pricer.sample_integrand(prob, torch.from_numpy(j)).cpu().numpy()
        ref = cm.integrand(prob, j)
        scale = np.max(np.abs(ref))
        err = np.abs(got - ref)
        assert np.all(err <= 1e-13 * np.abs(ref) + 1e-15 * scale), (n, np.max(err / (np.abs(ref) + 1e-300)))


# ------------------------------------------------------------------ K3 ----
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_mpo_contracts_to_bitreversed_dft(pricer, n):
    cores = pricer.mpo(n, 1e-12)
    Q = tt.mpo_full(cores)
    ref = tt.qft_bitrev_dense(n)
    # rounding keeps ||Q - Q_n||_F <= tol ||Q_n||_F = tol sqrt(M)
    assert np.linalg.norm(Q - ref) <= 2e-12 * math.sqrt(1 << n)
    ranks = tt.tt_ranks(cores)
    assert max(ranks) <= 24


@pytest.mark.parametrize("n", [16, 28, 40])
def test_mpo_rank_and_unitarity_large_n(pricer, n):
    cores = pricer.mpo(n, 1e-12)
    ranks = tt.tt_ranks(cores)
    assert max(ranks) <= 24
    # ||Q x|| = ||x|| for random rank-2 inputs, checked through the apply path
    rng = np.random.default_rng(n)
    x = [rng.standard_normal((1 if s == 0 else 2, 2, 1 if s == n - 1 else 2))
         + 1j * rng.standard_normal((1 if s == 0 else 2, 2, 1 if s == n - 1 else 2)) for s in range(n)]
    y = pricer.tt_apply_qft(x, 1e-12)
    nx = math.sqrt(abs(tt_dot(x, x)))
    ny = math.sqrt(abs(tt_dot(y, y)))
    assert abs(nx - ny) <= 1e-10 * nx


def tt_dot(a, b):
    """<a, b> by the transfer-matrix contraction (any n)."""
    E = np.ones((1, 1), dtype=np.complex128)
    for A, B in zip(a, b):
        E = np.einsum("ab,aic,bid->cd", E, np.conj(A), B)
    return E[0, 0]


@pytest.mark.parametrize("n", [20, 40])
def test_apply_closed_forms(pricer, n):
    M = 1 << n
    # delta_0 -> M^{-1/2} everywhere
    delta = [np.array([1.0, 0.0], dtype=np.complex128).reshape(1, 2, 1) for _ in range(n)]
    y = pricer.tt_apply_qft(delta, 1e-12)
    rng = np.random.default_rng(1)
    for u in rng.integers(0, M, 8):
        assert abs(tt.tt_entry(y, bits_of(int(u), n)) - M ** -0.5) <= 1e-10 * M ** -0.5
    # plane wave exp(2 pi i m j / M) (rank 1, site l weight 2^(n-l)) -> sqrt(M) delta_{u,m}
    m = int(rng.integers(0, M))
    wave = []
    for l in range(1, n + 1):
        ph = 2.0 * math.pi * ((m << (n - l)) % M) / M
        wave.append(np.array([1.0, np.exp(1j * ph)]).reshape(1, 2, 1))
    y = pricer.tt_apply_qft(wave, 1e-12)
    assert abs(tt.tt_entry(y, bits_of(m, n)) - math.sqrt(M)) <= 1e-9 * math.sqrt(M)
    for u in list(rng.integers(0, M, 6)) + [(m + 1) % M, (m - 1) % M]:
        if int(u) != m:
            assert abs(tt.tt_entry(y, bits_of(int(u), n))) <= 1e-9 * math.sqrt(M)
    # geometric exp(gamma j): y_u = M^{-1/2} (1 - e^{gamma M}) / (1 - e^{gamma - 2 pi i u / M})
    gamma = -3.0 / M + 1j * 0.37
    geo = []
    for l in range(1, n + 1):
        geo.append(np.array([1.0, np.exp(gamma * (1 << (n - l)))]).reshape(1, 2, 1))
    y = pricer.tt_apply_qft(geo, 1e-12)
    nrm = math.sqrt(abs(tt_dot(geo, geo)))
    for u in rng.integers(0, M, 8):
        ref = M ** -0.5 * (1 - np.exp(gamma * M)) / (1 - np.exp(gamma - 2j * math.pi * int(u) / M))
        assert abs(tt.tt_entry(y, bits_of(int(u), n)) - ref) <= 1e-10 * nrm


# ------------------------------------------------------------------ K5 ----
def test_round_matches_truncated_svd(pricer):
    rng = np.random.default_rng(9)
    n = 9
    x = np.arange(1 << n) / (1 << n)
    f = (np.exp(-2 * x) * np.cos(7 * x) + 0.1j * x ** 3).reshape((2,) * n)
    base = tt.tt_svd(f, 1e-14)
    infl = []
    for k, G in enumerate(base):
        r0, d, r1 = G.shape
        if k == 0:
            H = np.concatenate([0.25 * G, 0.75 * G], axis=2)
        elif k == n - 1:
            H = np.concatenate([G, G], axis=0)
        else:
            H = np.zeros((2 * r0, d, 2 * r1), dtype=np.complex128)
            H[:r0, :, :r1] = G
            H[r0:, :, r1:] = G
        infl.append(H)
    for eps in (1e-12, 1e-6, 1e-3):
        out = pricer.tt_round(infl, eps)
        ref = tt.tt_round(infl, eps)
        assert tt.tt_ranks(out) == tt.tt_ranks(ref)
        assert np.linalg.norm(tt.tt_full(out) - f) <= eps * np.linalg.norm(f) * 1.01 + 1e-14
    # a full-rank random tensor (d = 4 exercises the MPO layout)
    A = rng.standard_normal((4,) * 5) + 1j * rng.standard_normal((4,) * 5)
    full = tt.tt_svd(A, 0.0)
    for eps in (1e-12, 0.1, 0.3):
        out = pricer.tt_round(full, eps)
        assert np.linalg.norm(tt.tt_full(out) - A) <= eps * np.linalg.norm(A) * 1.001
        assert tt.tt_ranks(out) == tt.tt_ranks(tt.tt_round(full, eps))


# --------------------------------------------------------------- K1+K2 ----
@pytest.mark.parametrize("prob", [wl.config1_gbm(), wl.config2_heston(16),
                                  wl.paper_grid_bs(12), wl.paper_grid_bs(16),
                                  wl.Problem(cf.MERTON, MODELS[cf.MERTON], r=0.02, T=0.5, n=14),
                                  wl.Problem(cf.VG, MODELS[cf.VG], r=0.02, T=2.0, n=15)])
def test_integrand_tt_matches_dense(pricer, prob):
    cores = pricer.integrand_tt(prob)
    got = tt.tt_full(cores).reshape(-1)
    ref = cm.integrand(prob, np.arange(1 << prob.n))
    assert np.linalg.norm(got - ref) <= 3 * prob.tol * np.linalg.norm(ref) + 1e-15
    assert max(tt.tt_ranks(cores)) <= 32


def _heavy_vg(n):
    """Variance-Gamma instances of the batch with slowly decaying integrand
    (small T/nu): their support exceeds the TT-SVD block, so the cross
    builder takes them."""
    b = wl.config3_batch()
    return [q.replace(n=n) for q in b if q.model == wl.VG and q.T / q.p[1] < 0.6][:2]


@pytest.mark.parametrize("n", [16, 20, 22])
def test_cross_builder_matches_dense(pricer, n):
    for q in _heavy_vg(n):
        cores = pricer.integrand_tt(q)
        got = tt.tt_full(cores).reshape(-1)
        ref = cm.integrand(q, np.arange(1 << n))
        assert np.linalg.norm(got - ref) <= 5 * q.tol * np.linalg.norm(ref), (q, n)
        assert max(tt.tt_ranks(cores)) <= 32


def test_cross_builder_sampled_entries_large_n(pricer):
    rng = np.random.default_rng(34)
    for q in _heavy_vg(34):
        cores = pricer.integrand_tt(q)
        nrm = math.sqrt(abs(tt_dot(cores, cores)))
        M = 1 << q.n
        js = np.unique(np.concatenate([np.arange(64), rng.integers(0, M, 64),
                                       (2.0 ** rng.uniform(6, 34, 64)).astype(np.int64)]))
        js = js[js < M]
        ref = cm.integrand(q, js)
        got = np.array([tt.tt_entry(cores, [(int(j) >> (q.n - 1 - s)) & 1 for s in range(q.n)]) for j in js])
        assert np.max(np.abs(got - ref)) <= 5 * q.tol * nrm


# ---------------------------------------------------------- K4+K5 on x ----
@pytest.mark.parametrize("n", [4, 9, 13])
def test_apply_matches_dense_dft(pricer, n):
    prob = wl.config2_heston(n).replace(eta=0.25 * 2 ** (16 - n))
    x = cm.integrand(prob, np.arange(1 << n))
    cores = tt.tt_svd(x.reshape((2,) * n), 1e-14)
    y = pricer.tt_apply_qft(cores, 1e-12)
    got = tt.tt_full(y).reshape(-1)  # index = sum_l mu_l 2^(n-l) = bitrev(u)
    ref = cm.fft_radix2(x)[tt.bitrev(np.arange(1 << n), n)]
    # rows of tt_full are read site 1 first: position bitrev(u) holds y_u
    assert np.linalg.norm(got - ref) <= 5e-12 * np.linalg.norm(x)


# ------------------------------------------------------------- prices -----
def check_prices(pricer, probs, sample=12, seed=0, tol=PRICE_TOL, J=None, require_ok=True):
    strikes = [cm.strike_window(p) for p in probs]
    prices, logk, status, info = pricer.price_batch(probs, strikes, raise_on_error=False)
    prices = prices.cpu().numpy()
    logk = logk.cpu().numpy()
    rng = np.random.default_rng(seed)
    off = 0
    worst = 0.0
    for p, (lb, st, q), s in zip(probs, strikes, status):
        u = wl.strike_set(lb, st, q)
        if require_ok:
            assert s == 0, (p, s, pricer.last_error())
        if s == 0:
            pick = np.unique(np.concatenate([[0, q - 1, q // 2], rng.integers(0, q, sample)]))
            c_ref, k_ref = cm.prices(p, u[pick], route="sparse", J=J)
            err = np.max(np.abs(prices[off + pick] - c_ref))
            worst = max(worst, err / p.S0)
            assert err <= tol * p.S0, (p, err)
            assert np.max(np.abs(logk[off:off + q] - (math.log(p.S0) + cm.log_moneyness(p, u)))) < 1e-12
        else:
            assert np.all(np.isnan(prices[off:off + q]))
        off += q
    return worst, status, info


def test_config1_prices_and_black_scholes(pricer):
    p = wl.config1_gbm()
    worst, _, _ = check_prices(pricer, [p], sample=64)
    lb, st, q = cm.strike_window(p)
    prices, logk, _, _ = pricer.price_batch([p], [(lb, st, q)])
    K = np.exp(logk.cpu().numpy())
    bs = cfm.bs_call(p.S0, K, p.r, 0.2, p.T)
    assert np.max(np.abs(prices.cpu().numpy() - bs)) <= 1e-8 * p.S0


@pytest.mark.parametrize("n", [16, 20, 24, 28, 32, 36, 40])
def test_config2_heston_sweep(pricer, n):
    check_prices(pricer, [wl.config2_heston(n)], sample=10, seed=n)


def test_paper_grid_nrmse_floor(pricer):
    floor = 3.1e-13  # printed SFFT floor of Sec. 4.1
    for n in (10, 14, 16):
        p = wl.paper_grid_bs(n)
        M = 1 << n
        prices, logk, status, _ = pricer.price_batch([p], [(0, 1, M)] if M <= 65536 else None)
        c = prices.cpu().numpy()
        lk = logk.cpu().numpy()
        e, cnt = cm.nrmse(p, c, lk, lambda K: cfm.bs_call(100.0, K, 0.05, 0.3, 0.5))
        assert cnt > 0 and e < 30 * floor, (n, e)
        # element-wise parity inside the evaluation window K in [50, 150]; outside
        # it exp(-alpha k) reaches ~1e12 and amplifies rounding (Sec. 4)
        c_ref, _ = cm.prices_from_y(p, np.arange(M), cm.y_full(p, "fft"))
        K = np.exp(lk)
        win = (K >= 50.0) & (K <= 150.0)
        assert np.max(np.abs(c[win] - c_ref[win])) <= PRICE_TOL * p.S0


def test_config3_sample(pricer):
    batch = wl.config3_batch()
    # 2 instances per model spread over n, plus the largest n present
    picks = []
    for model in (wl.HESTON, wl.MERTON, wl.VG):
        idx = [i for i, p in enumerate(batch) if p.model == model]
        idx.sort(key=lambda i: batch[i].n)
        picks += [idx[0], idx[len(idx) // 2], idx[-1]]
    probs = [batch[i] for i in picks]
    # every picked instance must price; the oracle checks those whose direct
    # sum runs over at most 2^22 points
    strikes = [cm.strike_window(p) for p in probs]
    _, _, status, _ = pricer.price_batch(probs, strikes, raise_on_error=False)
    assert status == [0] * len(probs), status
    sel = [p for p in probs if cm.support_limit(p) <= (1 << 22)]
    check_prices(pricer, sel, sample=6, seed=3)


def test_config4_accuracy_at_tol_1e7(pricer):
    # the mixed batch at n = 30 with truncation tolerance 1e-7 (the mixed-
    # precision configuration's accuracy target, 1e-6 S0 per instance), on
    # the FP64 path: every instance prices, and sampled strikes of those whose
    # direct sum runs over at most 2^20 points agree with the oracle
    probs = wl.config3_batch(48, n_lo=30, n_hi=30, tol=1e-7)
    strikes = [cm.strike_window(p) for p in probs]
    _, _, status, info = pricer.price_batch(probs, strikes, raise_on_error=False)
    assert status == [0] * len(probs), status
    sel = [p for p in probs if cm.support_limit(p) <= (1 << 20)]
    assert len(sel) >= 24
    worst, _, _ = check_prices(pricer, sel, sample=8, seed=4, tol=1e-6)
    assert worst <= 1e-6


def test_out_of_bounds_prices_are_flagged(pricer):
    # Heston near its moment explosion of order alpha + 1 = 2.5 (kappa 0.52,
    # sigma_v 0.92, rho -0.17, T 2.73): the damped integrand is far sharper
    # than the grid, and the discrete Carr-Madan sum itself (the oracle's,
    # too) leaves the no-arbitrage bounds. The pricer returns SFFT_EBOUNDS
    # with the prices written; an ordinary instance in the same call is 0.
    from paper_2607_28435_b300 import sfft
    bad = wl.heston_surrogate_batch(16384, 260728435)[8441]
    good = wl.config2_heston(16)
    probs = [bad, good]
    strikes = [cm.strike_window(p, qmax=256) for p in probs]
    prices, logk, status, _ = pricer.price_batch(probs, strikes, raise_on_error=False)
    assert status == [sfft.SFFT_EBOUNDS, 0], status
    c = prices.cpu().numpy()
    lb, st, q = strikes[0]
    assert np.all(np.isfinite(c[:q]))
    u = wl.strike_set(lb, st, q)
    pick = np.array([0, q // 2, q - 1])
    ref, _ = cm.prices(bad, u[pick], route="sparse")
    assert np.max(np.abs(c[pick] - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert np.max(ref) > bad.S0


def test_reused_batch_matches_lists(pricer):
    # a Batch marshalled once gives the same prices, statuses and ranks as the
    # list form, on two calls in a row
    from paper_2607_28435_b300 import sfft
    probs = wl.config3_batch(24)
    strikes = [cm.strike_window(p) for p in probs]
    p0, k0, s0, i0 = pricer.price_batch(probs, strikes, raise_on_error=False)
    b = sfft.Batch(probs, strikes)
    for _ in range(2):
        p1, k1, s1, i1 = pricer.price_batch(b, None, raise_on_error=False)
        assert list(s1) == s0
        assert list(i1) == i0
        assert np.array_equal(p1.cpu().numpy(), p0.cpu().numpy())
        assert np.array_equal(k1.cpu().numpy(), k0.cpu().numpy())


def test_heavy_tail_prices(pricer):
    # cross-built integrands priced end to end; oracle over the full grid
    probs = _heavy_vg(20)
    check_prices(pricer, probs, sample=8, seed=5, J=1 << 20)


def test_whole_batch_prices(pricer):
    # every instance of the 4096-instance batch prices (finite, status OK)
    # except the few whose discrete Carr-Madan sum itself leaves the
    # no-arbitrage bounds (near a moment explosion at alpha = 1.5): those are
    # flagged SFFT_EBOUNDS, and the oracle's sum breaks the bound there too
    from paper_2607_28435_b300 import sfft
    batch = wl.config3_batch()
    strikes = [cm.strike_window(p) for p in batch]
    prices, logk, status, _ = pricer.price_batch(batch, strikes, raise_on_error=False)
    assert bool(torch.isfinite(prices).all())
    assert set(status) <= {0, sfft.SFFT_EBOUNDS}, sorted(set(status))
    flagged = [i for i, s in enumerate(status) if s != 0]
    assert len(flagged) <= 8, flagged
    c, lk = prices.cpu().numpy(), logk.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([q for _, _, q in strikes])])
    for i in flagged[:3]:
        p = batch[i]
        lb, st, q = strikes[i]
        ci, ki = c[offs[i]:offs[i + 1]], lk[offs[i]:offs[i + 1]] - math.log(p.S0)
        lower = np.maximum(p.S0 * (1 - np.exp(ki) * math.exp(-p.r * p.T)), 0.0)
        band = 1e-6 * p.S0 * np.maximum(1.0, np.exp(-p.alpha * ki))
        j = int(np.argmax(np.maximum(lower - ci, ci - p.S0) - band))
        ref, _ = cm.prices(p, wl.strike_set(lb, st, q)[[j]], route="sparse")
        assert abs(ref[0] - ci[j]) <= 1e-8 * p.S0
        assert ref[0] < lower[j] - band[j] or ref[0] > p.S0 + band[j], (i, ref[0], lower[j])


# -------------------------------------------------------------- dense -----
@pytest.mark.parametrize("prob", [wl.config1_gbm(), wl.config2_heston(16), wl.config2_heston(22),
                                  wl.paper_grid_bs(12),
                                  wl.Problem(cf.VG, MODELS[cf.VG], r=0.02, T=2.0, n=17)])
def test_dense_baseline(pricer, prob):
    strikes = [cm.strike_window(prob)]
    prices, logk, status, _ = pricer.dense_price_batch([prob], strikes)
    lb, st, q = strikes[0]
    u = wl.strike_set(lb, st, q)
    c = prices.cpu().numpy()
    if prob.n <= 16:
        c_ref, _ = cm.prices_from_y(prob, u, cm.y_full(prob, "fft")[u])
        assert np.max(np.abs(c - c_ref)) <= 1e-10 * prob.S0
    else:
        pick = np.unique(np.concatenate([[0, q - 1], np.random.default_rng(2).integers(0, q, 14)]))
        c_ref, _ = cm.prices(prob, u[pick], J=1 << prob.n)
        assert np.max(np.abs(c[pick] - c_ref)) <= 1e-10 * prob.S0


# -------------------------------------------------------------- errors ----
def test_invalid_inputs_are_rejected(pricer):
    from paper_2607_28435_b300 import sfft
    good = wl.config1_gbm()
    lb, st, q = cm.strike_window(good, qmax=16)
    bad = [good.replace(n=0), good.replace(S0=float("nan")), good.replace(tol=0.0),
           good.replace(eta=-1.0), good.replace(model=7), good.replace(max_rank=99)]
    for b in bad:
        with pytest.raises(sfft.SfftError) as ei:
            pricer.price_batch([b], [(lb, st, q)])
        assert ei.value.status == sfft.SFFT_EINVAL
    # bad strike sets
    for s in ((lb, 3, q), (lb + 1, st * 2, q), (0, 1, 1 << 13), (1 << 12, 1, 1)):
        with pytest.raises(sfft.SfftError) as ei:
            pricer.price_batch([good], [s])
        assert ei.value.status == sfft.SFFT_EINVAL
    # VG moment of order alpha+1 infinite: EMOMENT, NaN prices, batch continues
    vg_bad = wl.Problem(cf.VG, (0.4, 0.5, -0.3), alpha=8.0, n=12)
    prices, _, status, _ = pricer.price_batch([vg_bad, good], [(lb, st, q), (lb, st, q)],
                                              raise_on_error=False)
    assert status == [sfft.SFFT_EMOMENT, 0]
    c = prices.cpu().numpy()
    assert np.all(np.isnan(c[:q])) and np.all(np.isfinite(c[q:]))


def _heston_explosion_ode(kappa, sv, rho, p, tmax):
    """Moment-explosion time by integrating the Riccati equation of the v0
    coefficient, B' = p(p-1)/2 + (rho sv p - kappa) B + sv^2 B^2 / 2, until B
    passes 1e8 (independent of the closed form the library uses)."""
    from scipy.integrate import solve_ivp
    f = lambda t, B: [0.5 * p * (p - 1) + (rho * sv * p - kappa) * B[0] + 0.5 * sv * sv * B[0] ** 2]
    ev = lambda t, B: B[0] - 1e8
    ev.terminal = True
    r = solve_ivp(f, [0, tmax], [0.0], events=ev, rtol=1e-10, atol=1e-12, max_step=0.01)
    return r.t_events[0][0] if len(r.t_events[0]) else math.inf


def test_heston_moment_check_matches_riccati(pricer):
    from paper_2607_28435_b300 import sfft
    cases = [(1.1129, 0.0347, 0.6659, -0.021, 0.0653), (0.528, 0.0239, 0.535, -0.1916, 0.0336),
             (0.5, 0.04, 1.0, 0.0, 0.04), (2.0, 0.04, 0.9, -0.9, 0.04), (0.3, 0.04, 1.2, 0.5, 0.04)]
    for par in cases:
        tstar = _heston_explosion_ode(par[0], par[2], par[3], 2.5, 40.0)
        for T in (0.5 * tstar, 1.2 * tstar) if math.isfinite(tstar) else (3.0,):
            q = wl.Problem(cf.HESTON, par, r=0.02, T=T, alpha=1.5, n=12)
            _, _, status, _ = pricer.price_batch([q], [cm.strike_window(q, qmax=8)], raise_on_error=False)
            want = sfft.SFFT_EMOMENT if T > tstar else 0
            assert status == [want], (par, T, tstar, status)


def test_empty_batch_and_zero_strikes(pricer):
    prices, logk, status, _ = pricer.price_batch([], [])
    assert status == []
    good = wl.config1_gbm()
    prices, logk, status, _ = pricer.price_batch([good], [(0, 1, 0)])
    assert status == [0]
