"""Python binding of the C ABI in include/sfft.h (ctypes, argument marshalling
only). Device buffers are torch CUDA tensors; every computation runs in the
CUDA library. There is no fallback: if libsfft.so is missing or no CUDA device
is present, the calls raise.
"""
from __future__ import annotations

import collections.abc
import ctypes
import math
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfft.so")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

(SFFT_OK, SFFT_EINVAL, SFFT_EMOMENT, SFFT_ENOMEM, SFFT_ECUDA, SFFT_ERANK, SFFT_ENOCONV, SFFT_ETIMEOUT,
 SFFT_EBOUNDS) = range(9)
STATUS_NAMES = ["OK", "EINVAL", "EMOMENT", "ENOMEM", "ECUDA", "ERANK", "ENOCONV", "ETIMEOUT", "EBOUNDS"]
MAX_N = 48
NPHASES = 10
PHASE_NAMES = ["probe", "build", "zipup", "round", "readout", "mpo", "dense_sample", "dense_fft",
               "dense_gather", "cross"]
PHASE_KERNELS = ["k_support_probe+k_build_lists", "k_integrand_ttsvd", "k_zipup", "k_tt_round", "k_readout",
                 "k_mpo_interp+k_tt_round", "k_dense_sample", "k_fft_pass", "k_dense_gather",
                 "k_integrand_cross+k_tt_round"]
PRECISION_FP64, PRECISION_MIXED = 0, 1
MAX_RANK = 32
MAX_STRIKES = 65536
DENSE_MAX_N = 32


class SfftProblem(ctypes.Structure):
    _fields_ = [("model", c_int32), ("quad", c_int32), ("n", c_int32), ("max_rank", c_int32),
                ("p", c_double * 8), ("S0", c_double), ("r", c_double), ("T", c_double),
                ("alpha", c_double), ("eta", c_double), ("tol", c_double), ("k0", c_double)]


class SfftInfo(ctypes.Structure):
    _fields_ = [("status", c_int32), ("int_rank", c_int32), ("mpo_rank", c_int32),
                ("out_rank", c_int32), ("tt_bytes", c_int64)]


MLP_MAX_LAYERS = 8


class SfftTune(ctypes.Structure):
    _fields_ = [("build_p", c_int32), ("round_r", c_int32), ("zip_ctas", c_int32)]

    def as_dict(self):
        return dict(build_p=self.build_p, round_r=self.round_r, zip_ctas=self.zip_ctas)


class SfftMlp(ctypes.Structure):
    """sfft_mlp of include/sfft_mlp.h: widths and device pointers per layer."""
    _fields_ = [("n_layers", c_int32), ("width", c_int32 * (MLP_MAX_LAYERS + 1)), ("mode", c_int32),
                ("w", c_void_p * MLP_MAX_LAYERS), ("b", c_void_p * MLP_MAX_LAYERS), ("tc_weights", c_void_p)]


MLP_TENSOR_CORES, MLP_CUDA_CORES = 0, 1


_P_MLP = ctypes.POINTER(SfftMlp)

EXPORTS = {
    "sfft_mlp_workspace_floats": (c_int64, [_P_MLP, c_int64]),
    "sfft_mlp_normalize": (c_int32, [c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p]),
    "sfft_mlp_forward": (c_int32, [_P_MLP, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sfft_mlp_mse_grad": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "sfft_mlp_backward": (c_int32, [_P_MLP, c_void_p, c_int64, c_void_p, c_void_p,
                                    ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_void_p, c_void_p]),
    "sfft_mlp_tc_timeouts": (c_int32, []),
    "sfft_mlp_pack_bytes": (c_int64, [_P_MLP]),
    "sfft_mlp_pack": (c_int32, [_P_MLP, c_void_p, c_void_p]),
    "sfft_mlp_adam": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, ctypes.c_float, c_int64, c_void_p]),
    "sfft_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32]),
    "sfft_destroy": (c_int32, [c_void_p]),
    "sfft_set_stream": (c_int32, [c_void_p, c_void_p]),
    "sfft_tier2_counts": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "sfft_set_precision": (c_int32, [c_void_p, c_int32]),
    "sfft_autotune": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_int32, ctypes.POINTER(c_int64),
                                ctypes.POINTER(c_int64), ctypes.POINTER(c_int32), c_void_p, c_void_p, c_int32,
                                ctypes.POINTER(SfftTune), ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "sfft_tune_lookup": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_int32, ctypes.POINTER(SfftTune),
                                   ctypes.POINTER(c_int32)]),
    "sfft_tune_key": (c_int32, [ctypes.POINTER(SfftProblem), c_int32, ctypes.c_char_p, c_int32]),
    "sfft_tune_export": (c_int32, [c_void_p, ctypes.c_char_p, c_int64, ctypes.POINTER(c_int64)]),
    "sfft_tune_import": (c_int32, [c_void_p, ctypes.c_char_p]),
    "sfft_tune_trials": (c_int32, [c_void_p, ctypes.POINTER(SfftTune), ctypes.POINTER(c_double), c_int32,
                                   ctypes.POINTER(c_int32)]),
    "sfft_strike_window": (c_int32, [ctypes.POINTER(SfftProblem), c_double, c_double, c_int32,
                                     ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                     ctypes.POINTER(c_int32)]),
    "sfft_price_batch": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_int32,
                                   ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                   ctypes.POINTER(c_int32), c_void_p, c_void_p,
                                   ctypes.POINTER(c_int32), ctypes.POINTER(SfftInfo)]),
    "sfft_dense_price_batch": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_int32,
                                         ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                         ctypes.POINTER(c_int32), c_void_p, c_void_p,
                                         ctypes.POINTER(c_int32), ctypes.POINTER(SfftInfo)]),
    "sfft_qft_price_batch": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_int32,
                                         ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                         ctypes.POINTER(c_int32), c_void_p, c_void_p,
                                         ctypes.POINTER(c_int32), ctypes.POINTER(SfftInfo)]),
    "sfft_graph_create": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_int32,
                                    ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                    ctypes.POINTER(c_int32), c_void_p, c_void_p,
                                    ctypes.POINTER(c_void_p)]),
    "sfft_graph_launch": (c_int32, [c_void_p, c_void_p]),
    "sfft_graph_update": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem)]),
    "sfft_graph_status": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(SfftInfo)]),
    "sfft_graph_last_error": (ctypes.c_char_p, [c_void_p]),
    "sfft_graph_destroy": (c_int32, [c_void_p]),
    "sfft_sample_integrand": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem), c_void_p, c_int64,
                                        c_void_p]),
    "sfft_integrand_tt": (c_int32, [c_void_p, ctypes.POINTER(SfftProblem),
                                    ctypes.POINTER(c_int32), c_void_p, c_int64]),
    "sfft_mpo": (c_int32, [c_void_p, c_int32, c_double, ctypes.POINTER(c_int32), c_void_p, c_int64]),
    "sfft_tt_round": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_int32), c_void_p,
                                c_double, c_int32, ctypes.POINTER(c_int32), c_void_p, c_int64]),
    "sfft_tt_apply_qft": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32), c_void_p, c_double,
                                    c_int32, ctypes.POINTER(c_int32), c_void_p, c_int64]),
    "sfft_profile_enable": (c_int32, [c_void_p, c_int32]),
    "sfft_profile_read": (c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                    ctypes.POINTER(c_double), ctypes.POINTER(c_int64), c_int32]),
    "sfft_calibrate_fp64": (c_int32, [c_void_p, ctypes.POINTER(c_double)]),
    "sfft_tt_round_noalloc": (c_int32, [c_int32, c_int32, ctypes.POINTER(c_int32), c_void_p, c_double,
                                        c_int32, ctypes.POINTER(c_int32), c_void_p, c_int64, c_void_p,
                                        ctypes.c_char_p, c_int32]),
    "sfft_status_string": (ctypes.c_char_p, [c_int32]),
    "sfft_last_error": (ctypes.c_char_p, [c_void_p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsfft.so and declare every exported symbol. Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_2607_28435_b300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Batch:
    """Problems and strike sets marshalled into the C arrays of sfft_price_batch,
    with the per-instance status and info arrays the call fills. Building one
    costs Python time proportional to the batch (tens of ms for 4096 problems);
    a caller that prices the same batch repeatedly builds it once. Lazy
    statuses()/infos() convert the filled arrays back to Python."""

    def __init__(self, problems, strikes):
        cnt = len(problems)
        n1 = max(cnt, 1)
        self.count = cnt
        self.problems = (SfftProblem * n1)(*[to_c_problem(p) for p in problems])
        self.l_begin = (c_int64 * n1)(*[int(s[0]) for s in strikes])
        self.stride = (c_int64 * n1)(*[int(s[1]) for s in strikes])
        self.q = (c_int32 * n1)(*[int(s[2]) for s in strikes])
        self.total = sum(int(s[2]) for s in strikes)
        self.status = (c_int32 * n1)()
        self.info = (SfftInfo * n1)()

    def statuses(self):
        return [self.status[i] for i in range(self.count)]

    def _info(self, i):
        return dict(status=self.info[i].status, int_rank=self.info[i].int_rank,
                    mpo_rank=self.info[i].mpo_rank, out_rank=self.info[i].out_rank)

    def infos(self):
        return [self._info(i) for i in range(self.count)]

    def status_view(self):
        return _View(self.count, lambda i: self.status[i])

    def info_view(self):
        return _View(self.count, self._info)


class _View(collections.abc.Sequence):
    """Read-only sequence over a filled C array, converting one entry per access."""

    def __init__(self, n, get):
        self._n, self._get = n, get

    def __len__(self):
        return self._n

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self._get(k) for k in range(*i.indices(self._n))]
        if i < 0:
            i += self._n
        if not 0 <= i < self._n:
            raise IndexError(i)
        return self._get(i)


class Graph:
    """A batch of fixed shape captured as a CUDA graph (sfft_graph_*): launch()
    replays it on the current torch stream, update() swaps in new problem
    statements of the same shape, status() reads the last replay's statuses.
    The prices and log_strikes tensors stay bound to the graph."""

    def __init__(self, pricer, problems, strikes):
        torch = pricer.torch
        self.lib = pricer.lib
        self.torch = torch
        self.batch = Batch(problems, strikes)
        dev = torch.device("cuda", pricer.device)
        n = max(self.batch.total, 1)
        self.prices = torch.empty(n, dtype=torch.float64, device=dev)
        self.log_strikes = torch.empty(n, dtype=torch.float64, device=dev)
        self.h = c_void_p()
        b = self.batch
        s = self.lib.sfft_graph_create(pricer.h, b.problems, b.count, b.l_begin, b.stride, b.q,
                                       c_void_p(_ptr(self.prices)), c_void_p(_ptr(self.log_strikes)),
                                       ctypes.byref(self.h))
        if s != SFFT_OK:
            raise SfftError(s, pricer.last_error())

    def _check(self, s):
        if s != SFFT_OK:
            raise SfftError(s, self.lib.sfft_graph_last_error(self.h).decode())

    def launch(self):
        stream = self.torch.cuda.current_stream().cuda_stream
        self._check(self.lib.sfft_graph_launch(self.h, c_void_p(stream)))

    def update(self, problems):
        arr = (SfftProblem * max(len(problems), 1))(*[to_c_problem(p) for p in problems])
        self._check(self.lib.sfft_graph_update(self.h, arr))

    def status(self, raise_on_error=False):
        b = self.batch
        s = self.lib.sfft_graph_status(self.h, b.status, b.info)
        if raise_on_error:
            self._check(s)
        return b.statuses(), b.infos()

    def close(self):
        if self.h:
            self.lib.sfft_graph_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SfftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def to_c_problem(prob) -> SfftProblem:
    """Marshal a workloads.Problem (or any object with the same attributes)."""
    c = SfftProblem()
    c.model = int(prob.model)
    c.quad = int(prob.quad)
    c.n = int(prob.n)
    c.max_rank = int(getattr(prob, "max_rank", 0))
    p = list(prob.p) + [0.0] * (8 - len(prob.p))
    for i in range(8):
        c.p[i] = float(p[i])
    c.S0, c.r, c.T, c.alpha = float(prob.S0), float(prob.r), float(prob.T), float(prob.alpha)
    c.eta, c.tol = float(prob.eta), float(prob.tol)
    c.k0 = float(getattr(prob, "k0", math.nan))
    return c


def strike_window(prob, lo: float = -1.5, hi: float = 1.5, qmax: int = 4096) -> Tuple[int, int, int]:
    lib = load_library()
    lb, st, q = c_int64(), c_int64(), c_int32()
    cp = to_c_problem(prob)
    s = lib.sfft_strike_window(ctypes.byref(cp), lo, hi, qmax, ctypes.byref(lb), ctypes.byref(st),
                               ctypes.byref(q))
    if s != SFFT_OK:
        raise SfftError(s, lib.sfft_status_string(s).decode())
    return lb.value, st.value, q.value


def tune_key(problems) -> str:
    """The batch part of the tuning signature (host only)."""
    lib = load_library()
    arr = (SfftProblem * max(len(problems), 1))(*[to_c_problem(p) for p in problems])
    buf = ctypes.create_string_buffer(256)
    s = lib.sfft_tune_key(arr, len(problems), buf, 256)
    if s != SFFT_OK:
        raise SfftError(s, "sfft_tune_key")
    return buf.value.decode()


def _ptr(t) -> int:
    return t.data_ptr() if t is not None else 0


class Pricer:
    """One library context on one CUDA device. All device work runs on the
    torch current stream at call time."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the SFFT pricer needs a CUDA device")
        self.torch = torch
        self.lib = load_library()
        self.device = device
        h = c_void_p()
        s = self.lib.sfft_create(ctypes.byref(h), device)
        if s != SFFT_OK:
            raise SfftError(s, "sfft_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.sfft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ------------------------------------------------------------
    def _stream(self):
        st = self.torch.cuda.current_stream(self.device).cuda_stream
        self.lib.sfft_set_stream(self.h, c_void_p(st))

    def _check(self, s: int):
        if s != SFFT_OK:
            raise SfftError(s, self.lib.sfft_last_error(self.h).decode())

    def profile(self, on: bool = True):
        self._check(self.lib.sfft_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, reset: bool = True):
        ms = (c_double * NPHASES)()
        fl = (c_double * NPHASES)()
        ev = (c_double * NPHASES)()
        ln = (c_int64 * NPHASES)()
        self._check(self.lib.sfft_profile_read(self.h, ms, fl, ev, ln, 1 if reset else 0))
        return {PHASE_NAMES[i]: dict(ms=ms[i], flops=fl[i], evals=ev[i], launches=ln[i])
                for i in range(NPHASES)}

    def calibrate_fp64(self) -> float:
        g = c_double()
        self._stream()
        self._check(self.lib.sfft_calibrate_fp64(self.h, ctypes.byref(g)))
        return g.value

    def last_error(self) -> str:
        return self.lib.sfft_last_error(self.h).decode()

    def autotune(self, problems, strikes=None, reps: int = 2):
        """Time the batch under the candidate first-tier carves (sfft_autotune);
        returns (chosen configuration dict, ms chosen, ms default)."""
        torch = self.torch
        b = problems if isinstance(problems, Batch) else Batch(problems, strikes)
        dev = torch.device("cuda", self.device)
        pr = torch.empty(max(b.total, 1), dtype=torch.float64, device=dev)
        lk = torch.empty_like(pr)
        cfg, t1, t0 = SfftTune(), c_double(), c_double()
        self._stream()
        self._check(self.lib.sfft_autotune(self.h, b.problems, b.count, b.l_begin, b.stride, b.q,
                                           c_void_p(_ptr(pr)), c_void_p(_ptr(lk)), reps, ctypes.byref(cfg),
                                           ctypes.byref(t1), ctypes.byref(t0)))
        return cfg.as_dict(), t1.value, t0.value

    def tune_trials(self):
        """[(configuration dict, ms)] of the last autotune, in the order timed."""
        cfgs = (SfftTune * 16)()
        ms = (c_double * 16)()
        n = c_int32()
        self._check(self.lib.sfft_tune_trials(self.h, cfgs, ms, 16, ctypes.byref(n)))
        return [(cfgs[i].as_dict(), ms[i]) for i in range(min(n.value, 16))]

    def tune_lookup(self, problems):
        arr = (SfftProblem * max(len(problems), 1))(*[to_c_problem(p) for p in problems])
        cfg, found = SfftTune(), c_int32()
        self._check(self.lib.sfft_tune_lookup(self.h, arr, len(problems), ctypes.byref(cfg), ctypes.byref(found)))
        return cfg.as_dict(), bool(found.value)

    def tune_export(self) -> str:
        n = c_int64()
        self._check(self.lib.sfft_tune_export(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        self._check(self.lib.sfft_tune_export(self.h, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()

    def tune_import(self, text: str):
        self._check(self.lib.sfft_tune_import(self.h, text.encode()))

    def set_precision(self, mixed: bool):
        """FP64 everywhere (False, the default) or the MPO contraction in
        complex FP32 on the tensor cores (True); see sfft_set_precision."""
        self._check(self.lib.sfft_set_precision(self.h, PRECISION_MIXED if mixed else PRECISION_FP64))

    def tier2_counts(self):
        """Instances the last pricing call's first-tier launches handed to their
        second tier: dict with keys build, cross, zipup, round."""
        c = (c_int32 * 4)()
        self._stream()
        self._check(self.lib.sfft_tier2_counts(self.h, c))
        return dict(build=c[0], cross=c[1], zipup=c[2], round=c[3])

    # -- pricing ------------------------------------------------------------
    def _price(self, fn, problems, strikes, prices=None, log_strikes=None, raise_on_error=True):
        torch = self.torch
        b = problems if isinstance(problems, Batch) else Batch(problems, strikes)
        cnt, tot = b.count, b.total
        dev = torch.device("cuda", self.device)
        if prices is None:
            prices = torch.empty(max(tot, 1), dtype=torch.float64, device=dev)
        if log_strikes is None:
            log_strikes = torch.empty(max(tot, 1), dtype=torch.float64, device=dev)
        self._stream()
        s = fn(self.h, b.problems, cnt, b.l_begin, b.stride, b.q, c_void_p(_ptr(prices)),
               c_void_p(_ptr(log_strikes)), b.status, b.info)
        if raise_on_error and s not in (SFFT_OK,):
            self._check(s)
        if b is problems:  # a reused Batch: hand back its arrays, converted on access
            return prices[:tot], log_strikes[:tot], b.status_view(), b.info_view()
        return prices[:tot], log_strikes[:tot], b.statuses(), b.infos()

    def price_batch(self, problems, strikes=None, prices=None, log_strikes=None, raise_on_error=True):
        """TT-SFFT prices. strikes: list of (l_begin, stride, q) per problem; or pass a
        Batch as `problems` (strikes=None) to reuse its marshalled arrays."""
        return self._price(self.lib.sfft_price_batch, problems, strikes, prices, log_strikes,
                           raise_on_error)

    def dense_price_batch(self, problems, strikes, prices=None, log_strikes=None,
                          raise_on_error=True):
        """Dense-FFT Carr-Madan baseline prices, same contract."""
        return self._price(self.lib.sfft_dense_price_batch, problems, strikes, prices, log_strikes,
                           raise_on_error)

    def qft_price_batch(self, problems, strikes=None, prices=None, log_strikes=None,
                        raise_on_error=True):
        """QFT route by exact statevector emulation (|amplitude| readout), same contract."""
        return self._price(self.lib.sfft_qft_price_batch, problems, strikes, prices, log_strikes,
                           raise_on_error)

    # -- single steps -------------------------------------------------------
    def sample_integrand(self, prob, j):
        torch = self.torch
        j = j.to(device=torch.device("cuda", self.device), dtype=torch.int64).contiguous()
        x = torch.empty(j.numel(), dtype=torch.complex128, device=j.device)
        cp = to_c_problem(prob)
        self._stream()
        self._check(self.lib.sfft_sample_integrand(self.h, ctypes.byref(cp), c_void_p(_ptr(j)),
                                                   j.numel(), c_void_p(_ptr(x))))
        return x

    def _alloc_cores(self, n, d):
        cap = n * d * MAX_RANK * MAX_RANK
        return self.torch.empty(cap, dtype=self.torch.complex128,
                                device=self.torch.device("cuda", self.device)), cap

    def integrand_tt(self, prob):
        cores, cap = self._alloc_cores(prob.n, 2)
        ranks = (c_int32 * (MAX_N + 1))()
        cp = to_c_problem(prob)
        self._stream()
        self._check(self.lib.sfft_integrand_tt(self.h, ctypes.byref(cp), ranks, c_void_p(_ptr(cores)), cap))
        return unpack(cores, [ranks[i] for i in range(prob.n + 1)], 2)

    def mpo(self, n, tol):
        cores, cap = self._alloc_cores(n, 4)
        ranks = (c_int32 * (MAX_N + 1))()
        self._stream()
        self._check(self.lib.sfft_mpo(self.h, n, tol, ranks, c_void_p(_ptr(cores)), cap))
        return unpack(cores, [ranks[i] for i in range(n + 1)], 4)

    def tt_round(self, cores: List, tol: float, max_rank: int = 0):
        n = len(cores)
        d = cores[0].shape[1]
        flat, ranks = pack(cores, self.torch, self.device)
        out, cap = self._alloc_cores(n, d)
        rin = (c_int32 * (MAX_N + 1))(*ranks)
        rout = (c_int32 * (MAX_N + 1))()
        self._stream()
        self._check(self.lib.sfft_tt_round(self.h, n, d, rin, c_void_p(_ptr(flat)), tol, max_rank, rout,
                                           c_void_p(_ptr(out)), cap))
        return unpack(out, [rout[i] for i in range(n + 1)], d)

    def tt_apply_qft(self, cores: List, tol: float, max_rank: int = 0):
        n = len(cores)
        flat, ranks = pack(cores, self.torch, self.device)
        out, cap = self._alloc_cores(n, 2)
        rin = (c_int32 * (MAX_N + 1))(*ranks)
        rout = (c_int32 * (MAX_N + 1))()
        self._stream()
        self._check(self.lib.sfft_tt_apply_qft(self.h, n, rin, c_void_p(_ptr(flat)), tol, max_rank, rout,
                                               c_void_p(_ptr(out)), cap))
        return unpack(out, [rout[i] for i in range(n + 1)], 2)


def tt_round_noalloc(cores: List, tol: float, max_rank: int = 0, device: int = 0):
    """Round a TT with the allocation-free entry point (no context; the
    library's static device scratch). Input/output device buffers are
    allocated here by torch, which is the caller's side of the contract."""
    import torch
    lib = load_library()
    n = len(cores)
    d = cores[0].shape[1]
    flat, ranks = pack(cores, torch, device)
    cap = n * d * MAX_RANK * MAX_RANK
    out = torch.empty(cap, dtype=torch.complex128, device=torch.device("cuda", device))
    width = max(MAX_N + 1, len(ranks))
    rin = (c_int32 * width)(*ranks)
    rout = (c_int32 * width)()
    err = ctypes.create_string_buffer(256)
    with torch.cuda.device(device):
        st = torch.cuda.current_stream(device).cuda_stream
        s = lib.sfft_tt_round_noalloc(n, d, rin, c_void_p(flat.data_ptr()), tol, max_rank, rout,
                                      c_void_p(out.data_ptr()), cap, c_void_p(st), err, 256)
    if s != SFFT_OK:
        raise SfftError(s, err.value.decode())
    return unpack(out, [rout[i] for i in range(n + 1)], d)


def unpack(flat, ranks: Sequence[int], d: int):
    """Packed device cores -> list of host numpy arrays (r0, d, r1)."""
    host = flat.cpu().numpy()
    out, o = [], 0
    for s in range(len(ranks) - 1):
        sz = ranks[s] * d * ranks[s + 1]
        out.append(host[o:o + sz].reshape(ranks[s], d, ranks[s + 1]).copy())
        o += sz
    return out


def pack(cores, torch, device):
    ranks = [1] + [int(G.shape[2]) for G in cores]
    flat = np.concatenate([np.asarray(G, dtype=np.complex128).reshape(-1) for G in cores])
    return torch.from_numpy(flat).to(torch.device("cuda", device)), ranks
