"""TT rounding (Sec. 3.1, Oseledets 2011) on random tensors with decaying
separable structure: A = sum_k w_k (x) v_(k,s), w_k = 10^(-k c), given as a TT
with redundant ranks (every core duplicated into a block-diagonal pair). The
rounding must meet the Frobenius bound ||A - A~|| <= eps ||A|| and keep ranks
within one of the plain truncated-SVD rounding of the oracle, on both
physical dimensions the path uses (d = 2 for price TTs, d = 4 for operators)."""
import numpy as np
import pytest

from oracle import tt

torch = pytest.importorskip("torch")
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


def _separable(rng, n, d, K, decay):
    full = np.zeros((d,) * n, dtype=np.complex128)
    for k in range(K):
        term = np.array(1.0 + 0j)
        for _ in range(n):
            v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
            term = np.multiply.outer(term, v / np.linalg.norm(v))
        full = full + 10.0 ** (-decay * k) * term
    return full


def _inflate(cores):
    out = []
    n = len(cores)
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
        out.append(H)
    return out


@pytest.mark.parametrize("seed", range(8))
def test_round_random_separable(pricer, seed):
    rng = np.random.default_rng(1000 + seed)
    d = 2 if seed % 2 == 0 else 4
    n = 8 if d == 2 else 6
    K = int(rng.integers(4, 13))
    decay = float(rng.uniform(0.3, 1.5))
    full = _separable(rng, n, d, K, decay)
    cores = _inflate(tt.tt_svd(full, 1e-14))
    nrm = np.linalg.norm(full)
    for eps in (1e-12, 1e-8, 1e-4):
        out = pricer.tt_round(cores, eps)
        err = np.linalg.norm(tt.tt_full(out) - full)
        assert err <= eps * nrm * 1.01 + 1e-14 * nrm, (seed, eps, err / nrm)
        r_out, r_ref = tt.tt_ranks(out), tt.tt_ranks(tt.tt_round(cores, eps))
        assert all(a <= b + 1 for a, b in zip(r_out, r_ref)), (seed, eps, r_out, r_ref)
        assert sum(r_out) <= sum(r_ref) + 2, (seed, eps, r_out, r_ref)
