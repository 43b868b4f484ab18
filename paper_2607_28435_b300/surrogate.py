"""Price surrogate: a GELU multilayer perceptron fitted to SFFT prices over a
parameter box, answering repeated queries much faster than pricing each one,
with the SFFT pricer as the fallback outside the box or when the fit is not
accurate enough. It is not part of the paper's method (which builds the
pricing map as a tensor network, Sec. 3).

Inputs (8): the five Heston parameters (kappa, theta, sigma_v, rho, v0), r,
T and the log-moneyness k = log(K / S0); the box is workloads.SURROGATE_LO/HI.
Output: C / S0. Weights are kept in float32 for Adam and in bfloat16 for the
products, which accumulate in float32 (include/sfft_mlp.h). Every step runs in
the CUDA library; this module marshals pointers and drives the loop.
"""
from __future__ import annotations

import ctypes
import math
import time
from typing import List, Sequence, Tuple

import numpy as np

from . import sfft, workloads as wl

c_void_p = ctypes.c_void_p


def _ptr(t) -> int:
    return t.data_ptr()


class MLP:
    """Parameters in one flat float32 buffer [W_1, b_1, W_2, b_2, ...] (each W_l
    row-major w_l x w_{l-1}), its bfloat16 image for the products, the
    gradient buffer of the same layout and Adam's two moment buffers."""

    def __init__(self, widths: Sequence[int] = (8, 256, 256, 256, 256, 1), seed: int = 0, device: int = 0,
                 tensor_cores=None):
        import torch
        self.torch = torch
        self.lib = sfft.load_library()
        if len(widths) - 1 > sfft.MLP_MAX_LAYERS or widths[-1] != 1:
            raise ValueError("widths: at most 8 layers, one output")
        self.widths = tuple(int(w) for w in widths)
        self.L = len(widths) - 1
        self.dev = torch.device("cuda", device)
        # Glorot-uniform weights, zero biases, from a seeded generator
        rng = np.random.Generator(np.random.PCG64(seed))
        chunks, self.w_off, self.b_off = [], [], []
        off = 0
        for l in range(self.L):
            fi, fo = self.widths[l], self.widths[l + 1]
            a = math.sqrt(6.0 / (fi + fo))
            chunks.append(rng.uniform(-a, a, size=fo * fi))
            self.w_off.append(off)
            off += fo * fi
            chunks.append(np.zeros(fo))
            self.b_off.append(off)
            off += fo
        self.count = off
        self.p = torch.tensor(np.concatenate(chunks), dtype=torch.float32, device=self.dev)
        self.p16 = torch.empty(self.count, dtype=torch.int16, device=self.dev)
        self.g = torch.zeros_like(self.p)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.step = 0
        self.refresh_bf16()
        # products on the tensor cores (bfloat16 activations) when the shape
        # allows it and the caller did not ask otherwise, else CUDA cores
        if tensor_cores is None:
            tensor_cores = self.tc_shape_ok(self.widths)
        if tensor_cores and not self.tc_shape_ok(self.widths):
            raise ValueError("tensor-core products need w_0 <= 8 and hidden widths in 16..256, multiples of 16")
        self.tensor_cores = bool(tensor_cores)
        self.net = sfft.SfftMlp()
        self.net.mode = sfft.MLP_TENSOR_CORES if self.tensor_cores else sfft.MLP_CUDA_CORES
        self.net.n_layers = self.L
        for l in range(self.L + 1):
            self.net.width[l] = self.widths[l]
        for l in range(self.L):
            self.net.w[l] = _ptr(self.p16) + 2 * self.w_off[l]
            self.net.b[l] = _ptr(self.p) + 4 * self.b_off[l]
        self.packed = None
        if self.tensor_cores:
            # the weights in the tensor cores' operand layout, rewritten after
            # every update of the bfloat16 image
            nb = int(self.lib.sfft_mlp_pack_bytes(ctypes.byref(self.net)))
            self.packed = torch.empty(max(nb, 16), dtype=torch.uint8, device=self.dev)
            self.net.tc_weights = _ptr(self.packed)
            self._pack()
        self.gw = (c_void_p * self.L)(*[_ptr(self.g) + 4 * o for o in self.w_off])
        self.gb = (c_void_p * self.L)(*[_ptr(self.g) + 4 * o for o in self.b_off])
        self._ws = {}

    @staticmethod
    def tc_shape_ok(widths) -> bool:
        """Shapes the tensor-core forward pass takes (include/sfft_mlp.h)."""
        return (len(widths) >= 3 and 1 <= widths[0] <= 8 and widths[-1] == 1
                and all(16 <= w <= 256 and w % 16 == 0 for w in widths[1:-1]))

    # -- helpers ------------------------------------------------------------
    def _stream(self):
        return c_void_p(self.torch.cuda.current_stream(self.dev).cuda_stream)

    def _check(self, s):
        if s != sfft.SFFT_OK:
            raise sfft.SfftError(s, self.lib.sfft_status_string(s).decode())

    def _buf(self, name, n):
        b = self._ws.get(name)
        if b is None or b.numel() < n:
            b = self.torch.empty(max(n, 1), dtype=self.torch.float32, device=self.dev)
            self._ws[name] = b
        return b

    def _pack(self):
        if self.packed is not None:
            self._check(self.lib.sfft_mlp_pack(ctypes.byref(self.net), c_void_p(_ptr(self.packed)),
                                               self._stream()))

    def refresh_bf16(self):
        """p16 <- bfloat16(p): an Adam step with learning rate 0 and zero
        gradients leaves p unchanged and writes its bfloat16 image."""
        if self.count:
            gz = self.torch.zeros_like(self.p)
            mz = self.torch.zeros_like(self.p)
            vz = self.torch.zeros_like(self.p)
            self._check(self.lib.sfft_mlp_adam(self.count, c_void_p(_ptr(self.p)), c_void_p(_ptr(self.p16)),
                                               c_void_p(_ptr(gz)), c_void_p(_ptr(mz)), c_void_p(_ptr(vz)),
                                               0.0, 0.9, 0.999, 1.0, 1, self._stream()))
            if getattr(self, "net", None) is not None:
                self._pack()

    def weights(self) -> Tuple[List[np.ndarray], List[np.ndarray]]:
        """Host copies (float64) of the bfloat16 weights the products use and
        of the biases."""
        p16 = self.p16.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
        wf = p16.view(np.float32).astype(np.float64)
        pf = self.p.cpu().numpy().astype(np.float64)
        W, b = [], []
        for l in range(self.L):
            fo, fi = self.widths[l + 1], self.widths[l]
            W.append(wf[self.w_off[l]:self.w_off[l] + fo * fi].reshape(fo, fi))
            b.append(pf[self.b_off[l]:self.b_off[l] + fo])
        return W, b

    # -- passes -------------------------------------------------------------
    def normalize(self, raw, lo=wl.SURROGATE_LO, hi=wl.SURROGATE_HI):
        """raw: (B, 8) float64 device tensor -> (x float32 (B, 8), in_box int32 (B,))."""
        torch = self.torch
        B = raw.shape[0]
        lo_d = torch.tensor(lo, dtype=torch.float64, device=self.dev)
        hi_d = torch.tensor(hi, dtype=torch.float64, device=self.dev)
        x = torch.empty((B, self.widths[0]), dtype=torch.float32, device=self.dev)
        ib = torch.empty(B, dtype=torch.int32, device=self.dev)
        self._check(self.lib.sfft_mlp_normalize(c_void_p(_ptr(raw)), B, self.widths[0], c_void_p(_ptr(lo_d)),
                                                c_void_p(_ptr(hi_d)), c_void_p(_ptr(x)), c_void_p(_ptr(ib)),
                                                self._stream()))
        return x, ib

    def forward(self, x, keep: bool = False):
        """y = network(x) for x (B, w_0) float32; keep=True fills the workspace
        a backward pass needs."""
        B = x.shape[0]
        y = self.torch.empty(B, dtype=self.torch.float32, device=self.dev)
        if keep:
            ws = self._buf("ws", int(self.lib.sfft_mlp_workspace_floats(ctypes.byref(self.net), B)))
            s = self.lib.sfft_mlp_forward(ctypes.byref(self.net), c_void_p(_ptr(x)), B, c_void_p(_ptr(y)),
                                          c_void_p(_ptr(ws)), None, self._stream())
        else:
            sc = self._buf("infer", 2 * B * max(self.widths[1:-1] or (1,)))
            s = self.lib.sfft_mlp_forward(ctypes.byref(self.net), c_void_p(_ptr(x)), B, c_void_p(_ptr(y)),
                                          None, c_void_p(_ptr(sc)), self._stream())
        self._check(s)
        return y

    def gradients(self, x, t):
        """Forward, mean squared error against t and backward; fills self.g.
        Returns (y, loss as a device float)."""
        B = x.shape[0]
        y = self.forward(x, keep=True)
        dy = self._buf("dy", B)
        loss = self._buf("loss", 1)
        self._check(self.lib.sfft_mlp_mse_grad(c_void_p(_ptr(y)), c_void_p(_ptr(t)), B, c_void_p(_ptr(dy)),
                                               c_void_p(_ptr(loss)), self._stream()))
        sc = self._buf("bwd", 2 * B * max(self.widths[1:-1] or (1,)))
        self._check(self.lib.sfft_mlp_backward(ctypes.byref(self.net), c_void_p(_ptr(x)), B,
                                               c_void_p(_ptr(self._ws["ws"])), c_void_p(_ptr(dy)), self.gw,
                                               self.gb, c_void_p(_ptr(sc)), self._stream()))
        return y, loss[:1]

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.step += 1
        self._check(self.lib.sfft_mlp_adam(self.count, c_void_p(_ptr(self.p)), c_void_p(_ptr(self.p16)),
                                           c_void_p(_ptr(self.g)), c_void_p(_ptr(self.m)),
                                           c_void_p(_ptr(self.v)), lr, beta1, beta2, eps, self.step,
                                           self._stream()))
        self._pack()

    def fit(self, x, t, epochs: int, batch: int = 4096, lr: float = 2e-3, lr_end: float = 2e-5):
        """Minibatch Adam over the rows of (x, t) in their stored order (the
        caller shuffles once), with the learning rate decayed geometrically
        from lr to lr_end. Returns the last epoch's mean loss."""
        n = x.shape[0]
        steps = epochs * max(1, n // batch)
        decay = (lr_end / lr) ** (1.0 / max(1, steps - 1))
        k, acc = 0, None
        for _ in range(epochs):
            acc = self.torch.zeros(1, dtype=self.torch.float32, device=self.dev)
            nb = 0
            for s in range(0, n - batch + 1, batch):
                _, loss = self.gradients(x[s:s + batch], t[s:s + batch])
                self.adam(lr * decay ** k)
                acc += loss
                k += 1
                nb += 1
        return float(acc.item()) / max(nb, 1)


def sfft_dataset(pricer, problems, qmax: int = 4096, kmin: float = -1.5, kmax: float = 1.5):
    """Price every instance at the grid strikes with log-moneyness in
    [kmin, kmax] (at most qmax of them) with the SFFT pricer and return host
    arrays: raw query rows (count x 8: Heston parameters, r, T,
    log-moneyness) and targets C / S0."""
    strikes = [sfft.strike_window(p, kmin, kmax, qmax) for p in problems]
    # instances the pricer rejects (e.g. a Heston moment of order alpha + 1
    # that explodes before T) give no rows
    c, lk, st, _ = pricer.price_batch(problems, strikes, raise_on_error=False)
    c, lk = c.cpu().numpy(), lk.cpu().numpy()
    rows, tgt = [], []
    off = 0
    for p, (lb, sd, q), s in zip(problems, strikes, st):
        if s == 0 and q > 0:
            k = lk[off:off + q] - math.log(p.S0)
            base = np.array(list(p.p[:5]) + [p.r, p.T], dtype=np.float64)
            rows.append(np.concatenate([np.repeat(base[None, :], q, axis=0), k[:, None]], axis=1))
            tgt.append(c[off:off + q] / p.S0)
        off += q
    return np.concatenate(rows), np.concatenate(tgt)


class Surrogate:
    """A trained MLP and where to trust it. The box's (T, k) plane is cut into
    cells; a cell is trusted when the held-out maximum error of the prices in
    it is at most margin * accept * S0. Queries inside the box and in a
    trusted cell are priced by the network, all others by the SFFT pricer."""

    def __init__(self, pricer, mlp: MLP, cell_err: np.ndarray, accept: float = 1e-3, margin: float = 0.4,
                 S0: float = 100.0, n: int = 16, lo=wl.SURROGATE_LO, hi=wl.SURROGATE_HI):
        self.pricer, self.mlp = pricer, mlp
        self.cell_err = np.asarray(cell_err, dtype=np.float64)
        self.trusted_cells = self.cell_err <= margin * accept * S0
        self.trusted = bool(self.trusted_cells.any())
        self.S0, self.n, self.lo, self.hi = S0, n, lo, hi

    @staticmethod
    def cells(raw: np.ndarray, lo, hi, shape) -> Tuple[np.ndarray, np.ndarray]:
        """(T, k) cell of every row: the T and k ranges of the box cut into
        shape[0] and shape[1] equal parts."""
        iT = np.floor((raw[:, 6] - lo[6]) / (hi[6] - lo[6]) * shape[0]).astype(np.int64)
        ik = np.floor((raw[:, 7] - lo[7]) / (hi[7] - lo[7]) * shape[1]).astype(np.int64)
        return np.clip(iT, 0, shape[0] - 1), np.clip(ik, 0, shape[1] - 1)

    def price(self, raw: np.ndarray):
        """raw: (B, 8) host rows (Heston parameters, r, T, log-moneyness).
        Returns (prices, used_network mask, status): status is 0 for a
        network answer and the SFFT status of the query's fallback instance
        otherwise (for example SFFT_EMOMENT, whose price is NaN, or
        SFFT_EBOUNDS, whose price left the no-arbitrage bounds)."""
        torch = self.mlp.torch
        rd = torch.tensor(np.ascontiguousarray(raw, dtype=np.float64), device=self.mlp.dev)
        x, ib = self.mlp.normalize(rd, self.lo, self.hi)
        y = self.mlp.forward(x)
        out = (y.double() * self.S0).cpu().numpy()
        iT, ik = self.cells(raw, self.lo, self.hi, self.trusted_cells.shape)
        use = ib.cpu().numpy().astype(bool) & self.trusted_cells[iT, ik]
        status = np.zeros(len(raw), dtype=np.int32)
        miss = np.nonzero(~use)[0]
        if len(miss):
            out[miss], status[miss] = self.sfft_prices(raw[miss])
        return out, use, status

    def sfft_prices(self, raw: np.ndarray, max_span: int = sfft.MAX_STRIKES):
        """SFFT prices at the grid strike nearest to each query's
        log-moneyness, and each query's status (its instance's sfft status).
        Queries with the same seven model and market coordinates (an option
        chain) share one instance, priced over the contiguous grid range their
        strikes span when that is at most max_span points; every other query
        is an instance of its own."""
        M = 1 << self.n
        eta = 0.25
        dk = 2.0 * math.pi / (M * eta)
        k0 = -math.pi / eta
        u_all = np.clip(np.rint((raw[:, 7] - k0) / dk).astype(np.int64), 0, M - 1)
        groups = {}
        for i, row in enumerate(raw):
            groups.setdefault(tuple(float(v) for v in row[:7]), []).append(i)
        probs, strikes, picks = [], [], []
        for key, idx in groups.items():
            p = wl.Problem(wl.HESTON, key[:5], S0=self.S0, r=key[5], T=key[6], alpha=1.5, eta=eta, n=self.n,
                           quad=wl.SIMPSON_CM99)
            us = u_all[idx]
            lo_u, hi_u = int(us.min()), int(us.max())
            if len(idx) > 1 and hi_u - lo_u + 1 <= max_span:
                probs.append(p)
                strikes.append((lo_u, 1, hi_u - lo_u + 1))
                picks.append((idx, us - lo_u))
            else:
                for i, u in zip(idx, us):
                    probs.append(p)
                    strikes.append((int(u), 1, 1))
                    picks.append(([i], np.zeros(1, dtype=np.int64)))
        c, _, st, _ = self.pricer.price_batch(probs, strikes, raise_on_error=False)
        c = c.cpu().numpy()
        out = np.empty(len(raw))
        status = np.empty(len(raw), dtype=np.int32)
        off = 0
        for (idx, rel), (_, _, q), si in zip(picks, strikes, st):
            out[idx] = c[off + rel]
            status[idx] = si
            off += q
        return out, status


MARGINS = (0.3, 0.4, 0.5, 0.7, 1.0)


def train_surrogate(pricer, n_train_inst: int = 16384, n_test_inst: int = 1024, epochs: int = 12,
                    seed: int = 260728435, widths=(8, 256, 256, 256, 256, 1), lo=wl.SURROGATE_LO,
                    hi=wl.SURROGATE_HI, n: int = 16, accept: float = 1e-3, cells=(6, 12), qmax: int = 256,
                    margin=None, batch: int = 4096, lr: float = 2e-3):
    """SFFT prices of n_train_inst box instances at qmax strikes each (16384 x
    256 = 2^22 prices) train the network: many parameter sets with few strikes
    each, since the fit's error is set by how densely the seven model and
    market coordinates are sampled, not the strikes. Three further sets of
    n_test_inst instances, each drawn independently, then serve one purpose
    each:
      * held-out: the maximum error per (T, k) cell; a cell is trusted when it
        is at most margin * accept * S0;
      * validation: picks the margin (when margin is None), the largest of
        MARGINS whose trusted cells keep the validation maximum within
        accept * S0;
      * confirmation: untouched by either choice, it gives the reported share
        of queries the network answers and their maximum error.
    Returns (Surrogate, stats)."""
    torch = pricer.torch
    t0 = time.perf_counter()
    train = wl.heston_surrogate_batch(n_train_inst, seed, n=n, lo=lo, hi=hi)
    test = wl.heston_surrogate_batch(n_test_inst, seed + 1, n=n, lo=lo, hi=hi)
    val = wl.heston_surrogate_batch(n_test_inst, seed + 3, n=n, lo=lo, hi=hi)
    conf = wl.heston_surrogate_batch(n_test_inst, seed + 4, n=n, lo=lo, hi=hi)
    Xr, Y = sfft_dataset(pricer, train, qmax=qmax, kmin=lo[7], kmax=hi[7])
    perm = np.random.Generator(np.random.PCG64(seed + 2)).permutation(len(Y))
    Xr, Y = Xr[perm], Y[perm]
    t_data = time.perf_counter() - t0
    mlp = MLP(widths, seed=seed)
    x, _ = mlp.normalize(torch.tensor(Xr, device=mlp.dev), lo, hi)
    t = torch.tensor(Y, dtype=torch.float32, device=mlp.dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    last = mlp.fit(x, t, epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t1
    S0 = train[0].S0

    def errors(problems):
        Xh, Yh = sfft_dataset(pricer, problems, qmax=qmax, kmin=lo[7], kmax=hi[7])
        xh, _ = mlp.normalize(torch.tensor(Xh, device=mlp.dev), lo, hi)
        yh = mlp.forward(xh).double().cpu().numpy()
        return Xh, np.abs(yh - Yh) * S0

    Xh, eh = errors(test)
    iT, ik = Surrogate.cells(Xh, lo, hi, cells)
    cell_err = np.full(cells, np.inf)
    for a, b_, e in zip(iT, ik, eh):
        cell_err[a, b_] = e if not np.isfinite(cell_err[a, b_]) else max(cell_err[a, b_], e)
    Xv, ev = errors(val)
    vT, vk = Surrogate.cells(Xv, lo, hi, cells)
    # every margin on the validation set: share answered and maximum error
    by_margin = {}
    for mg in MARGINS:
        tm = (cell_err <= mg * accept * S0)[vT, vk]
        by_margin[str(mg)] = [float(tm.mean()), float(ev[tm].max()) if tm.any() else None]
    if margin is None:
        ok = [mg for mg in MARGINS if by_margin[str(mg)][1] is None or by_margin[str(mg)][1] <= accept * S0]
        margin = max(ok) if ok else min(MARGINS)
    sur = Surrogate(pricer, mlp, cell_err, accept=accept, margin=margin, S0=S0, n=n, lo=lo, hi=hi)
    # the confirmation set, independent of the held-out and validation sets
    Xc, ec = errors(conf)
    cT, ck = Surrogate.cells(Xc, lo, hi, cells)
    tc_ = sur.trusted_cells[cT, ck]
    stats = {"train_prices": int(len(Y)), "heldout_prices": int(len(eh)), "epochs": epochs,
             "final_loss": last, "heldout_max_abs_err": float(eh.max()),
             "heldout_rms_err": float(np.sqrt(np.mean(eh ** 2))),
             "trusted_cells": int(sur.trusted_cells.sum()), "cells": int(np.prod(cells)),
             "margin": margin, "validation_by_margin": by_margin,
             "confirm_prices": int(len(ec)), "confirm_trusted_fraction": float(tc_.mean()),
             "confirm_max_abs_err_trusted": float(ec[tc_].max()) if tc_.any() else None,
             "confirm_max_abs_err_all": float(ec.max()),
             "accept_abs": accept * S0, "tensor_cores": mlp.tensor_cores, "data_s": t_data, "fit_s": t_fit}
    return sur, stats


def main(argv=None):
    """Train on the full box and report the fit and the query rates as one
    JSON line: python -m paper_2607_28435_b300.surrogate [--instances N]
    [--epochs E] [--cells NT NK] (320 epochs: about three minutes on one B300)."""
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=16384)
    ap.add_argument("--qmax", type=int, default=256, help="strikes per training instance")
    ap.add_argument("--epochs", type=int, default=320)
    ap.add_argument("--cells", type=int, nargs=2, default=(6, 12), help="(T, k) cells of the trust table")
    ap.add_argument("--queries", type=int, default=1 << 20)
    ap.add_argument("--out", default=None, help="also write the JSON record to this file")
    ap.add_argument("--forward-only", type=int, default=0, metavar="PASSES",
                    help="no training: time PASSES forward passes of --queries rows through a randomly "
                         "initialised network of the surrogate's shape and print one JSON line")
    args = ap.parse_args(argv)
    if args.forward_only:
        mlp = MLP(seed=1)
        B = args.queries
        x = torch.rand(B, mlp.widths[0], device=mlp.dev) * 2 - 1
        mlp.forward(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.forward_only):
            mlp.forward(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.forward_only
        w = mlp.widths
        flops = 2.0 * B * sum(w[i] * w[i + 1] for i in range(len(w) - 1))
        print(json.dumps({"queries": B, "passes": args.forward_only, "ms": ms, "tflops": flops / ms / 1e9,
                          "tensor_cores": mlp.tensor_cores,
                          "timeouts": int(mlp.lib.sfft_mlp_tc_timeouts())}), flush=True)
        return
    pricer = sfft.Pricer(0)
    try:
        sur, st = train_surrogate(pricer, n_train_inst=args.instances, epochs=args.epochs,
                                  cells=tuple(args.cells), qmax=args.qmax)
        B = args.queries
        rng = np.random.Generator(np.random.PCG64(7))
        lo, hi = np.asarray(wl.SURROGATE_LO), np.asarray(wl.SURROGATE_HI)
        q = lo + (hi - lo) * rng.uniform(size=(B, 8))
        qd = torch.tensor(q, device=sur.mlp.dev)
        x, _ = sur.mlp.normalize(qd)
        sur.mlp.forward(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        reps = 5
        for _ in range(reps):
            x, _ = sur.mlp.normalize(qd)
            sur.mlp.forward(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        w = sur.mlp.widths
        flops = 2.0 * B * sum(w[i] * w[i + 1] for i in range(len(w) - 1))
        t0 = time.perf_counter()
        sur.sfft_prices(q[:4096])
        sfft_rate = 4096 / (time.perf_counter() - t0)
        # end to end: the network where trusted, one SFFT instance per other query
        Bs = min(B, 1 << 16)
        t0 = time.perf_counter()
        _, used, _ = sur.price(q[:Bs])
        torch.cuda.synchronize()
        served = Bs / (time.perf_counter() - t0)
        # option chains: 256 parameter sets x 256 strikes; SFFT alone prices
        # each chain as one instance, the surrogate answers trusted cells and
        # prices the rest of each chain as one instance
        nset, nk = 256, 256
        base = lo + (hi - lo) * rng.uniform(size=(nset, 8))
        ch = np.repeat(base, nk, axis=0)
        ch[:, 7] = np.tile(np.linspace(lo[7], hi[7], nk), nset)
        t0 = time.perf_counter()
        sur.sfft_prices(ch)
        chain_sfft = len(ch) / (time.perf_counter() - t0)
        t0 = time.perf_counter()
        _, used_ch, _ = sur.price(ch)
        torch.cuda.synchronize()
        chain_served = len(ch) / (time.perf_counter() - t0)
        out = {"surrogate": st, "queries": B, "network_queries_per_s": B / (ms * 1e-3),
               "network_ms": ms, "network_tflops": flops / (ms * 1e-3) / 1e12,
               "network_arithmetic": "tcgen05 bf16 (tensor cores)" if sur.mlp.tensor_cores else "fp32 CUDA cores",
               "sfft_one_instance_per_query_per_s": sfft_rate,
               "gain": B / (ms * 1e-3) / sfft_rate,
               "served": {"queries": Bs, "network_share": float(used.mean()), "queries_per_s": served,
                          "gain_over_sfft_alone": served / sfft_rate},
               "served_chains": {"queries": len(ch), "chains": nset, "network_share": float(used_ch.mean()),
                                 "queries_per_s": chain_served, "sfft_alone_queries_per_s": chain_sfft,
                                 "gain_over_sfft_alone": chain_served / chain_sfft}}
        print(json.dumps(out), flush=True)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(out, f, indent=1)
                f.write("\n")
    finally:
        pricer.close()


if __name__ == "__main__":
    main()
