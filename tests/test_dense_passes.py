"""The dense-FFT baseline's passes (Sec. 4.1's FFT route) on every digit
pattern they use: one pass of 2^R points for n <= 10 (radix-8 levels then a
radix-4 or radix-2 level, R mod 3 = 0, 1, 2), and two passes with several
columns per block (n = 11..20, the last pass taking several contiguous
sub-transforms per block). Every grid point (beyond 2^16 points every
2^(n-16)-th) is priced and compared with the
oracle's own FFT of the same samples (1e-10 S0, with the e^{-alpha k} growth
of the discrete sum's rounding at far strikes)."""
import numpy as np
import pytest

from oracle import carr_madan as cm
from paper_2607_28435_b300 import workloads as wl

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


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 13, 14, 16, 19, 20])
def test_every_grid_point(pricer, n):
    probs = [wl.config1_gbm().replace(n=n), wl.config2_heston(max(n, 2)).replace(n=n)]
    # every grid point up to the 65,536-strike limit, then a stride that covers the grid
    sd = 1 << max(0, n - 16)
    q = (1 << n) // sd
    for p in probs:
        prices, _, status, _ = pricer.dense_price_batch([p], [(0, sd, q)])
        assert list(status) == [0]
        c = prices.cpu().numpy()
        u = np.arange(q) * sd
        ref, _ = cm.prices_from_y(p, u, cm.y_full(p, "fft")[u])
        k = cm.log_moneyness(p, u)
        scale = p.S0 * np.maximum(1.0, np.exp(-p.alpha * k))
        assert np.all(np.abs(c - ref) <= 1e-10 * scale), (n, p.model)
