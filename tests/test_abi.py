"""C-ABI checks that need no GPU: the library builds and loads, exports every
function the headers in include/ declare, and its host-only helpers agree
with the oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import carr_madan as cm
from paper_2607_28435_b300 import build, sfft, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sfft.load_library()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(sfft_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(sfft.EXPORTS)


def test_struct_layout_matches_header():
    # sfft_problem: 4 int32, 8 doubles, 7 doubles
    assert ctypes.sizeof(sfft.SfftProblem) == 4 * 4 + 8 * 8 + 7 * 8
    assert ctypes.sizeof(sfft.SfftInfo) == 4 * 4 + 8
    # sfft_mlp: n_layers + 9 widths + mode (int32), 4 bytes of padding, then
    # 8 + 8 pointers and the packed-weight pointer
    assert ctypes.sizeof(sfft.SfftMlp) == 11 * 4 + 4 + 17 * 8
    assert sfft.SfftMlp.w.offset == 48
    assert sfft.SfftMlp.tc_weights.offset == 48 + 16 * 8


def test_status_strings(lib):
    for s in range(9):
        assert lib.sfft_status_string(s)
    assert b"unknown" in lib.sfft_status_string(99)


@pytest.mark.parametrize("prob", [wl.config1_gbm(), wl.config2_heston(16), wl.config2_heston(34),
                                  wl.config2_heston(40), wl.paper_grid_bs(12)])
def test_strike_window_matches_oracle(lib, prob):
    for lo, hi, qmax in ((-1.5, 1.5, 4096), (-0.3, 0.2, 100), (-1.5, 1.5, 1)):
        got = sfft.strike_window(prob, lo, hi, qmax)
        ref = cm.strike_window(prob, lo, hi, qmax)
        assert got == tuple(ref)
        lb, st, q = got
        assert st & (st - 1) == 0 and lb % st == 0 and q <= qmax


def test_strike_window_rejects_bad_problem(lib):
    p = wl.config1_gbm().replace(n=0)
    with pytest.raises(sfft.SfftError):
        sfft.strike_window(p)
    p = wl.config1_gbm().replace(eta=-1.0)
    with pytest.raises(sfft.SfftError):
        sfft.strike_window(p)
