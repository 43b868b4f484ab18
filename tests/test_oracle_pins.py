"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: values the
paper prints, closed forms, library routines, invariants, independent
formulations, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import carr_madan as cm
from oracle import cf, closed_forms as cfm, tt
from paper_2607_28435_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


PARAMS = {
    cf.GBM: (0.2,),
    cf.HESTON: wl.HESTON_CFG2,
    cf.MERTON: (0.2, 0.8, -0.1, 0.15),
    cf.VG: (0.2, 0.3, -0.14),
}


# ---------------------------------------------------------------- CF ------
@pytest.mark.parametrize("model", [cf.GBM, cf.HESTON, cf.MERTON, cf.VG])
def test_cf_normalisation_and_martingale(model):
    r, T = 0.03, 0.7
    p = PARAMS[model]
    assert abs(cf.phi1(model, p, r, T, np.array([0.0]))[0] - 1.0) < 1e-15
    # E[S_T/S0] = exp(rT): phi1(-i) = exp(rT)
    assert abs(cf.phi1(model, p, r, T, np.array([-1j]))[0] - math.exp(r * T)) < 1e-14
    # Hermitian symmetry of a characteristic function of a real variable
    v = np.linspace(-30, 30, 61)
    a = cf.phi1(model, p, r, T, v)
    b = cf.phi1(model, p, r, T, -v)
    assert np.max(np.abs(a - np.conj(b))) < 1e-14
    assert np.all(np.abs(a) <= 1.0 + 1e-14)


def test_cf_reductions_to_gbm():
    r, T, s = 0.04, 1.3, 0.25
    u = np.linspace(-20, 20, 81) - 1.7j
    gbm = cf.phi1(cf.GBM, (s,), r, T, u)
    # Merton with no jumps is GBM
    mer = cf.phi1(cf.MERTON, (s, 0.0, -0.2, 0.3), r, T, u)
    assert np.max(np.abs(mer - gbm)) < 1e-14
    # VG as nu -> 0 tends to GBM (error O(nu))
    vg = cf.phi1(cf.VG, (s, 1e-7, -0.2), r, T, np.linspace(-5, 5, 21) - 0.5j)
    gbm5 = cf.phi1(cf.GBM, (s,), r, T, np.linspace(-5, 5, 21) - 0.5j)
    assert np.max(np.abs(vg - gbm5)) < 1e-5
    # Heston with vanishing vol-of-vol and v0 = theta is GBM with sigma^2 = theta
    # (first order in sigma_v: the gap shrinks tenfold per tenfold smaller sigma_v)
    th = s * s
    gaps = []
    for sv in (1e-2, 1e-3, 1e-4, 1e-5):
        he = cf.phi1(cf.HESTON, (1.2, th, sv, -0.5, th), r, T, np.linspace(-5, 5, 21) - 0.5j)
        gaps.append(np.max(np.abs(he - gbm5)))
    assert gaps[-1] < 1e-5
    for a, b in zip(gaps[:-1], gaps[1:]):
        assert 8.0 < a / b < 12.0


# ------------------------------------------------------------ DFT routes --
def test_dft_routes_agree_and_match_library():
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 9):
        M = 1 << n
        x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        yd = cm.dft_direct(x)
        yf = cm.fft_radix2(x)
        ys = cm.sparse_sum(np.arange(M), x, np.arange(M), n)
        lib = np.fft.fft(x) / math.sqrt(M)
        scale = np.sum(np.abs(x))
        for y in (yd, yf, ys):
            assert np.max(np.abs(y - lib)) <= 1e-13 * scale
        # Parseval (unitarity of Eq. dft)
        assert abs(np.linalg.norm(yf) - np.linalg.norm(x)) <= 1e-13 * np.linalg.norm(x)


def test_sparse_sum_exact_phase_at_large_n():
    # a single spike x_j = delta_{j,j0}: y_u = M^{-1/2} exp(-2 pi i j0 u / M),
    # with j0*u far beyond 2^53 (the product wraps in uint64)
    n = 40
    j0 = (1 << 39) + 12345
    u = np.array([3, (1 << 38) + 7, (1 << 40) - 1], dtype=np.int64)
    y = cm.sparse_sum(np.array([j0]), np.array([1.0 + 0j]), u, n)
    t = [(j0 * int(uu)) % (1 << n) for uu in u]
    ref = np.exp(-2j * np.pi * np.array([float(tt_) for tt_ in t]) / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(y - ref)) < 1e-20


# ------------------------------------------------------- Black-Scholes ----
def test_config1_matches_black_scholes():
    p = wl.config1_gbm()
    g = cm.grid(p)
    u = np.arange(g["M"])
    for route in ("fft", "direct"):
        c, lk = cm.prices(p, u, route=route)
        K = np.exp(lk)
        sel = (K >= 50) & (K <= 150)
        bs = cfm.bs_call(p.S0, K[sel], p.r, 0.2, p.T)
        assert np.max(np.abs(c[sel] - bs)) <= 1e-8 * p.S0
    # the window |k'| <= 1.5 as well, by the direct sum at the window strikes
    lb, st, q = cm.strike_window(p)
    uu = wl.strike_set(lb, st, q)
    c, lk = cm.prices(p, uu, route="sparse")
    bs = cfm.bs_call(p.S0, np.exp(lk), p.r, 0.2, p.T)
    assert np.max(np.abs(c - bs)) <= 1e-8 * p.S0
    assert np.all(np.abs(lk - math.log(p.S0)) <= 1.5 + 1e-12)


def test_paper_grid_printed_nrmse():
    for n, val, how in _golden("paper_nrmse.txt"):
        n, val = int(n), float(val)
        p = wl.paper_grid_bs(n)
        g = cm.grid(p)
        u = np.arange(g["M"])
        y = cm.y_full(p, "direct")
        ref = lambda K: cfm.bs_call(100.0, K, 0.05, 0.3, 0.5)
        if how == "abs":
            c = cm.prices_qft_readout(p, u, y)
            lk = math.log(p.S0) + cm.log_moneyness(p, u)
        else:
            c, lk = cm.prices_from_y(p, u, y)
        e, cnt = cm.nrmse(p, c, lk, ref)
        assert cnt > 0
        # printed to three significant figures
        assert abs(e - val) <= 0.5e-2 * val + 0.005 * 10 ** math.floor(math.log10(val)), (n, e, val)


def test_paper_grid_fft_floor():
    floor = {r[0]: float(r[1]) for r in _golden("paper_floors.txt")}["fft"]
    for n in (12, 14, 16, 18):
        p = wl.paper_grid_bs(n)
        g = cm.grid(p)
        c, lk = cm.prices_from_y(p, np.arange(g["M"]), cm.y_full(p, "fft"))
        e, _ = cm.nrmse(p, c, lk, lambda K: cfm.bs_call(100.0, K, 0.05, 0.3, 0.5))
        # the printed floor is ~4.4e-15; allow a factor 30 for summation order
        assert e < 30 * floor, (n, e)


def test_put_call_parity_through_negative_damping():
    # alpha < -1 turns the same formula into put prices (the contour crosses
    # both poles of psi); C - P = S0 - K exp(-rT)
    for model in (cf.GBM, cf.HESTON, cf.MERTON, cf.VG):
        pc = wl.Problem(model, PARAMS[model], S0=100.0, r=0.05, T=1.0, alpha=1.5,
                        eta=0.25, n=12)
        pp = pc.replace(alpha=-2.5)
        lb, st, q = cm.strike_window(pc, qmax=64)
        u = wl.strike_set(lb, st, q)
        c, lk = cm.prices(pc, u)
        pu, _ = cm.prices(pp, u)
        K = np.exp(lk)
        lhs = c - pu
        rhs = pc.S0 - K * math.exp(-pc.r * pc.T)
        assert np.max(np.abs(lhs - rhs)) <= 1e-8 * pc.S0, model


def test_bs_put_matches_integral_of_the_payoff():
    # the put of the closed-form module against e^{-rT} E[max(K - S_T, 0)]
    # under the lognormal law of S_T, integrated numerically
    S0, r, sig, T = 100.0, 0.05, 0.25, 0.8
    mu = math.log(S0) + (r - 0.5 * sig * sig) * T
    sd = sig * math.sqrt(T)
    for K in (60.0, 95.0, 100.0, 130.0):
        def dens(s):
            return math.exp(-0.5 * ((math.log(s) - mu) / sd) ** 2) / (s * sd * math.sqrt(2 * math.pi))
        val, _ = integrate.quad(lambda s: (K - s) * dens(s), 1e-12, K, epsabs=1e-13, epsrel=1e-13,
                                limit=400)
        ref = math.exp(-r * T) * val
        assert abs(float(cfm.bs_put(S0, K, r, sig, T)) - ref) < 1e-10 * S0, K


def test_put_prices_through_negative_damping_match_bs_put():
    # the oracle's discrete sum with alpha < -1 prices puts; for GBM they are
    # the closed-form puts up to the discretisation error of config 1
    p = wl.Problem(cf.GBM, (0.2,), S0=100.0, r=0.05, T=1.0, alpha=-2.5, eta=0.25, n=12)
    lb, st, q = cm.strike_window(p, qmax=128)
    u = wl.strike_set(lb, st, q)
    c, lk = cm.prices(p, u)
    K = np.exp(lk)
    sel = (K >= 50.0) & (K <= 150.0)
    ref = cfm.bs_put(100.0, K[sel], 0.05, 0.2, 1.0)
    assert np.max(np.abs(c[sel] - ref)) <= 1e-8 * p.S0


def _support_cases():
    """Seeded draws of every model for the support-limit pin: eight per model
    from the mixed batch's boxes, plus the Heston and VG draws of that batch
    whose integrands decay slowest (largest support limit at n = 20)."""
    batch = wl.config3_batch(4096)
    rng = np.random.default_rng(20)
    out = [wl.Problem(cf.GBM, (s,), S0=100.0, r=0.025, T=T, alpha=1.5, eta=0.25, n=16)
           for s, T in ((0.1, 0.1), (0.2, 1.0), (0.4, 3.0), (0.15, 0.3))]
    for model in (cf.HESTON, cf.MERTON, cf.VG):
        idx = [i for i, p in enumerate(batch) if p.model == model]
        out += [batch[i] for i in rng.choice(idx, 8, replace=False)]
    # slowest decay among the first 600 Heston / VG draws whose support fits n = 20
    for model in (cf.HESTON, cf.VG):
        cands = [p.replace(n=20) for p in batch[:1800] if p.model == model]
        sup = [(cm.support_limit(p), k) for k, p in enumerate(cands)]
        sup = [t for t in sup if t[0] < (1 << 20)]
        sup.sort(reverse=True)
        out += [cands[k] for _, k in sup[:2]]
    return out


def test_support_limit_against_full_grid_sum():
    # the direct sum stops at support_limit(p); the sum over the whole grid
    # (own radix-2 FFT over all M points, J = M) must give the same prices
    # to 1e-11 S0 at every model, so no term that moves a price is dropped
    worst = 0.0
    for p0 in _support_cases():
        for n in (16, 18, 20):
            p = p0.replace(n=n)
            J = cm.support_limit(p)
            lb, st, q = cm.strike_window(p)
            u = wl.strike_set(lb, st, q)[::max(1, q // 48)]
            c_sup, _ = cm.prices(p, u, route="sparse", J=J)
            c_all, _ = cm.prices(p, u, route="fft")
            e = float(np.max(np.abs(c_sup - c_all))) / p.S0
            worst = max(worst, e)
            assert e <= 1e-11, (p.model, p.p, p.T, n, J, e)
    assert worst > 0.0


def test_support_limit_heston_branch_is_not_too_early():
    # Heston has no closed tail bound: the cut is the first dyadic block whose
    # samples are all negligible. The tail it drops, summed on the whole grid
    # beyond J, must be negligible too (and the block below J must not be)
    batch = wl.config3_batch(600)
    for p0 in [p for p in batch if p.model == cf.HESTON][:40]:
        p = p0.replace(n=20)
        J = cm.support_limit(p)
        if J >= (1 << 20):
            continue
        tail = np.sum(np.abs(cm.integrand(p, np.arange(J, 1 << 20, dtype=np.int64))))
        assert tail * math.exp(1.5 * 1.5) / math.pi * p.S0 <= 1e-11 * p.S0, (p.p, p.T, J, tail)


def test_merton_matches_poisson_series():
    s, lam, mu, dj = PARAMS[cf.MERTON]
    p = wl.Problem(cf.MERTON, (s, lam, mu, dj), S0=100.0, r=0.05, T=0.8, alpha=1.5,
                   eta=0.25, n=13)
    lb, st, q = cm.strike_window(p, qmax=200)
    u = wl.strike_set(lb, st, q)
    c, lk = cm.prices(p, u)
    ref = cfm.merton_call(p.S0, np.exp(lk), p.r, s, lam, mu, dj, p.T)
    assert np.max(np.abs(c - ref)) <= 1e-8 * p.S0


def _vg_gamma_mixture_call(S0, K, r, sigma, nu, theta, T):
    """VG call by conditioning on the gamma clock G ~ Gamma(T/nu, nu):
    given G = g the log-return is (r+omega)T + theta g + sigma sqrt(g) Z."""
    omega = math.log(1.0 - theta * nu - 0.5 * sigma * sigma * nu) / nu
    out = []
    for k in np.atleast_1d(K):
        def f(g):
            if g <= 0:
                return max(S0 * math.exp((r + omega) * T) - k, 0.0) * 0.0
            sg = sigma * math.sqrt(g)
            F = S0 * math.exp((r + omega) * T + theta * g + 0.5 * sg * sg)
            d1 = (math.log(F / k) + 0.5 * sg * sg) / sg
            d2 = d1 - sg
            cond = math.exp(-r * T) * (F * special.ndtr(d1) - k * special.ndtr(d2))
            dens = math.exp((T / nu - 1) * math.log(g) - g / nu - special.gammaln(T / nu) - (T / nu) * math.log(nu))
            return cond * dens
        val = 0.0
        edges = [0.0, 1e-6, 1e-3, 0.05, 0.3, 1.0, 3.0, 10.0, 60.0]
        for a, b in zip(edges[:-1], edges[1:]):
            val += integrate.quad(f, a, b, epsabs=1e-13, epsrel=1e-12, limit=400)[0]
        out.append(val)
    return np.array(out)


def test_vg_matches_gamma_mixture():
    s, nu, th = 0.2, 0.3, -0.14
    p = wl.Problem(cf.VG, (s, nu, th), S0=100.0, r=0.05, T=1.0, alpha=1.5,
                   eta=0.25, n=16)
    lb, st, q = cm.strike_window(p, lo=-0.4, hi=0.4, qmax=9)
    u = wl.strike_set(lb, st, q)
    c, lk = cm.prices(p, u)
    ref = _vg_gamma_mixture_call(p.S0, np.exp(lk), p.r, s, nu, th, p.T)
    assert np.max(np.abs(c - ref)) <= 1e-7 * p.S0


def _heston_1993_call(S0, K, r, T, kappa, theta, sv, rho, v0):
    """Heston's original two-probability formula (1993):
    C = S0 P1 - K exp(-rT) P2, P_j = 1/2 + 1/pi int_0^inf Re[exp(-i phi ln K) f_j / (i phi)]."""
    x = math.log(S0)
    a = kappa * theta

    def f(j, ph):
        uj = 0.5 if j == 1 else -0.5
        bj = kappa - rho * sv if j == 1 else kappa
        q = bj - rho * sv * ph * 1j
        d = np.sqrt(q * q - sv * sv * (2 * uj * ph * 1j - ph * ph))
        g = (q + d) / (q - d)
        ed = np.exp(d * T)
        C = r * ph * 1j * T + a / sv ** 2 * ((q + d) * T - 2.0 * np.log((1 - g * ed) / (1 - g)))
        D = (q + d) / sv ** 2 * (1 - ed) / (1 - g * ed)
        return np.exp(C + D * v0 + 1j * ph * x)

    out = []
    for k in np.atleast_1d(K):
        P = []
        for j in (1, 2):
            integrand_ = lambda ph: np.real(np.exp(-1j * ph * math.log(k)) * f(j, ph) / (1j * ph))
            val = integrate.quad(integrand_, 1e-12, 200.0, epsabs=1e-13, epsrel=1e-12, limit=1000)[0]
            P.append(0.5 + val / math.pi)
        out.append(S0 * P[0] - k * math.exp(-r * T) * P[1])
    return np.array(out)


def test_heston_matches_original_formulation():
    p = wl.config2_heston(16)
    lb, st, q = cm.strike_window(p, lo=-0.5, hi=0.5, qmax=9)
    u = wl.strike_set(lb, st, q)
    c, lk = cm.prices(p, u)
    ref = _heston_1993_call(p.S0, np.exp(lk), p.r, p.T, *wl.HESTON_CFG2)
    assert np.max(np.abs(c - ref)) <= 1e-7 * p.S0


def test_heston_discretisation_converges():
    # eta halved with M doubled keeps the strike spacing 2 pi/(M eta); the
    # grid start -pi/eta moves down by pi/eta_1, i.e. by M_1/2 points
    p1 = wl.config2_heston(16)
    p2 = p1.replace(eta=0.125, n=17)
    lb, st, q = cm.strike_window(p1, qmax=64)
    u1 = wl.strike_set(lb, st, q)
    c1, k1 = cm.prices(p1, u1)
    c2, k2 = cm.prices(p2, u1 + (1 << 15))
    assert np.max(np.abs(k1 - k2)) < 1e-12
    # eta = 0.25 is within ~2e-9 S0 of the converged integral (as for the
    # Black-Scholes pin), and the gap shrinks as eta is halved again
    d1 = np.max(np.abs(c1 - c2))
    assert d1 <= 1e-8 * p1.S0
    p3 = p1.replace(eta=0.0625, n=18)
    c3, _ = cm.prices(p3, u1 + (1 << 15) + (1 << 16))
    assert np.max(np.abs(c2 - c3)) < 0.5 * d1


def test_tail_bound_is_an_upper_bound():
    for model in (cf.GBM, cf.MERTON, cf.VG):
        p = wl.Problem(model, PARAMS[model], S0=100.0, r=0.025, T=0.4, alpha=1.5,
                       eta=0.25, n=18)
        J = 1 << 10
        j = np.arange(J, 1 << 18, dtype=np.int64)
        actual = np.sum(np.abs(cm.integrand(p, j)))
        bound = cm.tail_bound(p, J)
        assert actual <= bound * (1 + 1e-12), model
        env = cm.psi_envelope(p, 0.25 * j)
        psi = np.abs(cf.psi1(model, p.p, p.r, p.T, p.alpha, 0.25 * j))
        assert np.all(psi <= env * (1 + 1e-12) + 1e-300)


# -------------------------------------------------------------- tensors ---
def test_qft_operator_definition_and_product_form():
    for n in range(1, 8):
        A = tt.qft_bitrev_dense(n)
        B = tt.qft_bitrev_product_form(n)
        assert np.max(np.abs(A - B)) < 1e-13
        M = 1 << n
        F = np.fft.fft(np.eye(M), axis=0) / math.sqrt(M)
        assert np.max(np.abs(A[tt.bitrev(np.arange(M), n)] - F)) < 1e-13
        assert np.max(np.abs(A.conj().T @ A - np.eye(M))) < 1e-13


def test_tt_svd_exact_and_truncated():
    rng = np.random.default_rng(3)
    n = 10
    A = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).reshape((2,) * n)
    cores = tt.tt_svd(A, 0.0)
    assert np.max(np.abs(tt.tt_full(cores) - A)) < 1e-12
    for eps in (1e-1, 1e-3):
        c2 = tt.tt_svd(A, eps)
        err = np.linalg.norm(tt.tt_full(c2) - A)
        assert err <= eps * np.linalg.norm(A) * (1 + 1e-10)
    # closed-form ranks: exp is rank 1, sin is rank 2, a degree-3 polynomial rank 4
    x = np.arange(1 << n) / (1 << n)
    for f, rk in ((np.exp(3 * x), 1), (np.sin(5 * x), 2), (1 + x - 2 * x ** 2 + x ** 3, 4)):
        c = tt.tt_svd(f.reshape((2,) * n), 1e-13)
        assert max(tt.tt_ranks(c)) == rk
    # rank-one exponential TT of Sec. 3.3 equals exp(gamma x)
    g = -2.0 + 7.0j
    assert np.max(np.abs(tt.tt_full(tt.rank1_exp_tt(g, n)).reshape(-1) - np.exp(g * x))) < 1e-12


def test_tt_round_equals_truncated_svd():
    rng = np.random.default_rng(5)
    n = 9
    # a rank-3 tensor stored with inflated ranks (sum of a TT with itself minus a copy)
    base = tt.tt_svd((rng.standard_normal((2,) * n) + 0j), 0.0)
    x = np.arange(1 << n) / (1 << n)
    f = (np.exp(-x) + 0.3 * np.cos(4 * x)).reshape((2,) * n)
    cores = tt.tt_svd(f, 1e-14)
    # inflate: block-diagonal doubling with halves
    infl = []
    for k, G in enumerate(cores):
        r0, d, r1 = G.shape
        if k == 0:
            H = np.concatenate([0.5 * G, 0.5 * G], axis=2)
        elif k == n - 1:
            H = np.concatenate([G, G], axis=0)
        else:
            H = np.zeros((2 * r0, d, 2 * r1), dtype=np.complex128)
            H[:r0, :, :r1] = G
            H[r0:, :, r1:] = G
        infl.append(H)
    assert np.max(np.abs(tt.tt_full(infl) - f)) < 1e-12
    rounded = tt.tt_round(infl, 1e-12)
    assert tt.tt_ranks(rounded) == tt.tt_ranks(tt.tt_svd(f, 1e-12))
    assert np.linalg.norm(tt.tt_full(rounded) - f) <= 1e-12 * np.linalg.norm(f) * 1.01
    # on a random dense tensor, rounding with eps keeps the error below eps ||A||
    full_rank = tt.tt_svd(tt.tt_full(base), 0.0)
    r = tt.tt_round(full_rank, 0.2)
    assert np.linalg.norm(tt.tt_full(r) - tt.tt_full(base)) <= 0.2 * np.linalg.norm(tt.tt_full(base)) * 1.001


def test_mpo_full_index_convention():
    # build an MPO of Q_n by TT-SVD of its dense matrix with interleaved
    # (mu_l, lam_l) indices, then contract it back with mpo_full
    for n in (1, 2, 4, 5):
        Q = tt.qft_bitrev_dense(n)
        T = Q.reshape((2,) * (2 * n))  # rows mu_1..mu_n, cols lam_1..lam_n
        perm = [a for l in range(n) for a in (l, n + l)]
        T = T.transpose(perm).reshape((4,) * n)
        cores = tt.tt_svd(T, 1e-14)
        W = [G.reshape(G.shape[0], 2, 2, G.shape[2]) for G in cores]
        assert np.max(np.abs(tt.mpo_full(W) - Q)) < 1e-12


def test_tt_entry_matches_full_contraction():
    rng = np.random.default_rng(11)
    n = 7
    A = rng.standard_normal((2,) * n) + 1j * rng.standard_normal((2,) * n)
    cores = tt.tt_svd(A, 0.0)
    for idx in rng.integers(0, 2, size=(20, n)):
        assert abs(tt.tt_entry(cores, idx) - A[tuple(idx)]) < 1e-12
