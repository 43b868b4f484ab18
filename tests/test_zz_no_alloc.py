"""The allocation-free rounding entry point (sfft_tt_round_noalloc) against the
context-based sfft_tt_round, through the C ABI.

It serves callers that cannot allocate device memory at run time (their
memory manager owns the device, or cudaMalloc's implicit synchronisation is
not acceptable); its scratch is a static device array inside the library, so
two calls in a row must give the same result as the regular entry point even
though the second call finds the first call's data in that array. This file is
collected last so that a failure here does not hide other tests."""
import numpy as np
import pytest

from oracle import tt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inflated_tt(n, d, seed):
    """A low-rank tensor stored with doubled ranks (so rounding must cut)."""
    rng = np.random.default_rng(seed)
    x = np.arange(d ** n) / d ** n
    f = (np.exp(-3 * x) * np.cos(11 * x) + 0.2j * np.sin(5 * x) * x).reshape((d,) * n)
    f = f + 1e-3 * (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape))
    base = tt.tt_svd(f, 1e-13)
    out = []
    for k, G in enumerate(base):
        r0, dd, r1 = G.shape
        if k == 0:
            H = np.concatenate([0.5 * G, 0.5 * G], axis=2)
        elif k == n - 1:
            H = np.concatenate([G, G], axis=0)
        else:
            H = np.zeros((2 * r0, dd, 2 * r1), dtype=np.complex128)
            H[:r0, :, :r1] = G
            H[r0:, :, r1:] = G
        out.append(H)
    return out, f


@pytest.mark.parametrize("n,d,eps", [(9, 2, 1e-12), (9, 2, 1e-4), (5, 4, 1e-10)])
def test_noalloc_round_matches_context_round(n, d, eps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    cores, f = _inflated_tt(n, d, seed=n + d)
    if max(tt.tt_ranks(cores)) > sfft.MAX_RANK:
        pytest.skip("test tensor exceeds the rank cap")
    pricer = sfft.Pricer(0)
    try:
        ref = pricer.tt_round(cores, eps)
    finally:
        pricer.close()
    ref_full = tt.tt_full(ref)
    nrm = np.linalg.norm(f)
    for call in range(2):
        got = sfft.tt_round_noalloc(cores, eps)
        assert tt.tt_ranks(got) == tt.tt_ranks(ref), call
        # same algorithm and same arithmetic: agreement far inside the tolerance
        assert np.linalg.norm(tt.tt_full(got) - ref_full) <= 1e-12 * nrm, call
        assert np.linalg.norm(tt.tt_full(got) - tt.tt_full(cores)) <= eps * np.linalg.norm(tt.tt_full(cores)) * 1.01 + 1e-14


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_28435_b300 import build, sfft
    build.build()
    big = [np.ones((1, 2, 1), dtype=np.complex128)] * (sfft.MAX_N + 1)
    with pytest.raises((sfft.SfftError, ValueError)) as ei:
        sfft.tt_round_noalloc(big, 1e-12)
    assert "outside" in str(ei.value) or "n =" in str(ei.value)
