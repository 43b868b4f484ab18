#!/usr/bin/env python
"""Throughput of the batched TT-SFFT Carr-Madan pricer on one B300.

Metric: priced strikes per second. A step prices one seeded batch of pricing
instances (default: 4096 instances, one third each Heston / Merton / Variance-
Gamma, parameters drawn uniformly from the configured boxes, T in [0.1, 3],
grid exponent n uniform in 16..34, Simpson quadrature, eta = 0.25, alpha = 1.5,
tolerance 1e-12, FP64) at up to 4096 strikes each in |log(K/S0)| <= 1.5,
through the C ABI (sfft_price_batch): integrand TT build, zip-up MPO x TT
contraction with the cached Q_n operator, rounding and readout.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank prices its own seeded batch (weak scaling, no data
collectives); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one tier-1 k_zipup launch on the default
# 4096-instance batch, from a one-pass ncu capture of that launch
# (dram__bytes_read.sum 51,781,376 + dram__bytes_write.sum 916,991,232).
# The figure holds while the zip-up's code hashes to "src" (its part of
# tt_kernels.cu and the headers it uses); after any change to them the
# roofline reports traffic as null until it is captured again.
ZIPUP_TRAFFIC = {"bytes": 138172160 + 2354465792, "instances": 4096, "src": "24a203bf5d6a5c6c"}
KERNEL_SRCS = ("cplx.cuh", "kernels.cuh", "la.cuh", "model.cuh", "tc.cuh")
ZIPUP_REGION = ("// Mixed precision: the zip-up's MPO contraction", "// K6: readout")


def batch_problems(args, seed=None):
    """The mixed batch: n uniform in 16..34 at tol 1e-12 by default, or one n
    (--n) and another tolerance (--tol), e.g. --n 30 --tol 1e-7."""
    from paper_2607_28435_b300 import workloads as wl
    lo, hi = (args.n, args.n) if args.n else (16, 34)
    return wl.config3_batch(args.count, seed=wl.CONFIG3_SEED if seed is None else seed, n_lo=lo, n_hi=hi,
                            tol=args.tol)


def workload_name(args):
    nr = f"n {args.n}" if args.n else "n 16..34"
    tol = "" if args.tol == 1e-12 else f", tol {args.tol:g}"
    mixed = (", MPO contraction in complex FP32 on tcgen05 (QR/SVD FP64)"
             if getattr(args, "precision", "fp64") == "mixed" else "")
    return f"batched TT-SFFT, {args.count} instances (Heston/Merton/VG), {nr}{tol}{mixed}"


def kernel_src_hash():
    """Hash of the zip-up's code: its region of tt_kernels.cu and the headers."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2607_28435_b300", "csrc")
    for f in KERNEL_SRCS:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "tt_kernels.cu")) as fh:
        t = fh.read()
    a, b = t.index(ZIPUP_REGION[0]), t.index(ZIPUP_REGION[1])
    h.update(t[a:b].encode())
    return h.hexdigest()[:16]


METRIC = "priced strikes/s at <=1e-6*S0 err: batched TT-SFFT vs dense-FFT Carr-Madan, 1 B300"
UNIT = "strikes/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--n", type=int, default=None,
                    help="one grid exponent for every instance (default: uniform in 16..34)")
    ap.add_argument("--tol", type=float, default=1e-12, help="truncation tolerance of every instance")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the oracle check of a sample of the timed output")
    ap.add_argument("--no-config2", action="store_true",
                    help="skip the single-instance Heston sweep over n (TT-SFFT 16..40, dense 16..32)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default first-tier carves instead of tuning them for the batch first")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed: the zip-up's MPO contraction in complex FP32 on the tensor cores")
    return ap.parse_args()


# --------------------------------------------------------------------------- CPU oracle
def _oracle_task(args):
    """Price strikes lb + st*i (i < q) of one instance with the CPU oracle
    (direct sum at each strike)."""
    from oracle import carr_madan as cm
    from paper_2607_28435_b300 import workloads as wl
    prob, (lb, st, q) = args
    t0 = time.perf_counter()
    u = wl.strike_set(lb, st, q)
    cm.prices(prob, u, route="sparse")
    return q, time.perf_counter() - t0


def _oracle_prices_task(args):
    """Oracle prices (direct sum over the integrand support) of one instance
    at listed grid indices."""
    from oracle import carr_madan as cm
    import numpy as np
    prob, u = args
    c, _ = cm.prices(prob, np.asarray(u, dtype=np.int64), route="sparse")
    return c


def _support_task(prob):
    from oracle import carr_madan as cm
    return int(cm.support_limit(prob))


def accuracy_sample(pool, problems, strikes, status, prices, seed=17, per_cell=8, wide=48,
                    max_support=1 << 24, strikes_per_inst=8):
    """Check a seeded sample of one timed step's output against the oracle.

    The sample covers every (model, n) cell of the batch with up to
    `per_cell` instances (3 models x 19 grid exponents), plus `wide`
    instances whose integrand support exceeds 2^14 points (the ones the
    cross builder takes), each at `strikes_per_inst` strikes: both ends of
    its window and random ones. Instances whose direct sum would run over
    more than `max_support` points are left out and counted. prices: host
    array of the step's output. Returns the accuracy record of the bench line."""
    import numpy as np
    rng = np.random.default_rng(seed)
    offs = np.concatenate([[0], np.cumsum([s[2] for s in strikes])])
    sup = pool.map(_support_task, problems, chunksize=64)
    ok = [i for i, st in enumerate(status) if st == 0]
    cells = {}
    for i in ok:
        cells.setdefault((problems[i].model, problems[i].n), []).append(i)
    picks = []
    too_wide = 0
    for key in sorted(cells):
        idx = [i for i in cells[key] if sup[i] <= max_support]
        too_wide += len(cells[key]) - len(idx)
        picks += [int(i) for i in rng.permutation(idx)[:per_cell]]
    wide_all = [i for i in ok if sup[i] > (1 << 14)]
    wide_ok = [i for i in wide_all if sup[i] <= max_support and i not in set(picks)]
    picks += [int(i) for i in rng.permutation(wide_ok)[:wide]]
    tasks, where = [], []
    for i in picks:
        lb, st, q = strikes[i]
        k = np.unique(np.concatenate([[0, q - 1], rng.integers(0, q, max(strikes_per_inst - 2, 0))]))
        tasks.append((problems[i], (lb + st * k).tolist()))
        where.append(offs[i] + k)
    t0 = time.perf_counter()
    refs = pool.map(_oracle_prices_task, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    errs = np.array([float(np.max(np.abs(prices[w] - r))) / problems[i].S0
                     for i, w, r in zip(picks, where, refs)])
    models = sorted({problems[i].model for i in picks})
    return {"max_abs_err_over_S0": float(errs.max()) if len(errs) else None,
            "median_abs_err_over_S0": float(np.median(errs)) if len(errs) else None,
            "instances": len(picks), "strikes": int(sum(len(w) for w in where)),
            "over_1e-8": int((errs > 1e-8).sum()), "over_1e-6": int((errs > 1e-6).sum()),
            "n_covered": sorted({problems[i].n for i in picks}),
            "models_covered": models,
            "wide_support_instances": int(sum(1 for i in picks if sup[i] > (1 << 14))),
            "wide_support_in_batch": len(wide_all),
            "left_out_support_over": {"points": max_support, "instances": too_wide},
            "oracle_seconds": wall,
            "how": "after the timed steps: a seeded sample of the last timed step's device output, up "
                   f"to {per_cell} instances per (model, n) cell plus {wide} of the wide-support "
                   "(cross-built) instances, each at both ends of its window and random strikes, "
                   "against the oracle's FP64 direct sum over the integrand support"}


def _oracle_pieces(problems, strikes, skipped, seed=0):
    """Instances of the batch in a seeded random order, one piece each: its
    first max(32, 2^24 / support) strikes (all of them for small supports), so
    that no task runs much longer than a second. Instances whose support
    exceeds 2^20 points are counted in skipped[0] and left out (a direct sum
    there takes minutes per strike set). Yields (index, task)."""
    import numpy as np
    from oracle import carr_madan as cm
    for i in np.random.default_rng(seed).permutation(len(problems)):
        p, (lb, st, q) = problems[i], strikes[i]
        m = cm.support_limit(p)
        if m > (1 << 20):
            skipped[0] += 1
            continue
        yield int(i), (p, (lb, st, min(q, max(32, (1 << 24) // m))))


def oracle_sample(pool, problems, strikes, seconds, cores):
    """Time the oracle on a bounded sample of the batch. Each sampled instance
    prices one piece of its strikes; its whole cost is that piece's time
    scaled by its strike count (the direct sum costs the same at every strike
    of an instance). Workers take the next piece as soon as they are free,
    until about `seconds` of wall time (pieces in flight then finish).
    Returns (rate on the pool, rate on one core, instances, skipped, wall,
    strikes timed): one-core rate = sum q_i / sum t_i q_i / piece_i, and the
    pool's rate multiplies it by the concurrency the pool reached (summed
    piece seconds over wall)."""
    skipped = [0]
    it = _oracle_pieces(problems, strikes, skipped)
    t0 = time.perf_counter()
    pend = {}
    q_all = 0       # strikes of the sampled instances
    t_all = 0.0     # their estimated one-core seconds
    busy = 0.0      # summed piece seconds
    timed = 0       # strikes actually priced
    n_inst = 0

    def submit():
        nxt = next(it, None)
        if nxt is not None:
            i, task = nxt
            pend[pool.apply_async(_oracle_task, (task,))] = i

    for _ in range(cores):
        submit()
    while pend:
        ready = [r for r in pend if r.ready()]
        if not ready:
            time.sleep(0.002)
            continue
        for r in ready:
            i = pend.pop(r)
            qp, dt = r.get()
            q = strikes[i][2]
            q_all += q
            t_all += dt * q / qp
            busy += dt
            timed += qp
            n_inst += 1
            if time.perf_counter() - t0 < seconds:
                submit()
    wall = time.perf_counter() - t0
    one = q_all / t_all if t_all > 0 else 0.0
    return one * busy / wall, one, n_inst, skipped[0], wall, timed


def oracle_pool(ncores):
    """A spawned pool of `ncores` single-threaded workers: the thread-count
    variables are set before the spawn so that each worker's numpy starts with
    one thread and the pool does not oversubscribe the cores."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(ncores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


# --------------------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank, pool, ncores):
    import numpy as np
    import torch

    from paper_2607_28435_b300 import sfft, workloads as wl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    problems = batch_problems(args, seed=wl.CONFIG3_SEED + rank)
    strikes = [sfft.strike_window(p) for p in problems]
    total_q = sum(s[2] for s in strikes)
    pricer = sfft.Pricer(local_rank)
    mixed = args.precision == "mixed"
    pricer.set_precision(mixed)
    fp64_peak = pricer.calibrate_fp64()
    prices = torch.empty(total_q, dtype=torch.float64, device=dev)
    logk = torch.empty(total_q, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2
    # the problem and strike arrays are marshalled into C structs once; every
    # timed call passes them (host memory) through the C ABI
    batch = sfft.Batch(problems, strikes)

    status = None
    cold_ms = None
    for i in range(max(args.warmup, 0)):
        t0 = time.perf_counter()
        _, _, status, _ = pricer.price_batch(batch, None, prices, logk, raise_on_error=False)
        torch.cuda.synchronize()
        if i == 0:  # the first call of a fresh context also builds the batch's MPOs
            cold_ms = (time.perf_counter() - t0) * 1e3
    # tune the first-tier carves for this batch once, after the warm-up and
    # off the clock; the timed steps (and the graph) use the chosen ones
    tuning = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        chosen, ms_c, ms_d = pricer.autotune(batch, None, reps=2)
        tuning = {"chosen": chosen, "ms_chosen": ms_c, "ms_default": ms_d,
                  "trials": [dict(c, ms=m) for c, m in pricer.tune_trials()],
                  "default": {"build_p": 32, "round_r": 24, "zip_ctas": 0},
                  "tuning_s": time.perf_counter() - t0,
                  "how": "sfft_autotune: the batch timed (best of 2 calls, CUDA events) under the default carves "
                         "and by coordinate descent under zip_ctas 2, build_p 24 and 16, round_r 20 and 16; the "
                         "fastest is cached under the batch's signature"}

        _, _, status, _ = pricer.price_batch(batch, None, prices, logk, raise_on_error=False)
        torch.cuda.synchronize()

    # direct calls through the C ABI (problem arrays in host memory, marshalled
    # and uploaded inside each call), profiled: the phase times, flops and
    # launch counts of the kernels the graph below replays
    pricer.profile(True)
    pricer.profile_read(reset=True)
    torch.cuda.synchronize()
    direct_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, status, info = pricer.price_batch(batch, None, prices, logk, raise_on_error=False)
        e1.record()
        torch.cuda.synchronize()
        direct_ms.append(e0.elapsed_time(e1))
    prof = pricer.profile_read(reset=True)
    pricer.profile(False)
    q_direct = sum(s[2] for s, st in zip(strikes, status) if st == 0)
    direct = {"value": q_direct * args.steps / (sum(direct_ms) / 1e3), "unit": UNIT,
              "ms_per_step": sum(direct_ms) / args.steps,
              "how": "sfft_price_batch from the batch's host arrays each step (host planning and uploads "
                     "inside the call), profiled; the phase times and the roofline come from these calls"}

    # timed region: the step captured once as a CUDA graph (sfft_graph_*) with
    # its inputs resident in HBM, replayed; per-step CUDA events, L2 flushed
    # between steps, clocks sampled throughout
    g = sfft.Graph(pricer, problems, strikes)
    for _ in range(max(args.warmup, 1)):
        g.launch()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.launch()
        e1.record()
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    status, info = g.status()
    status = list(status)
    g_prices = g.prices

    ok = [s == 0 for s in status]
    q_ok = sum(s[2] for s, o in zip(strikes, ok) if o)
    # accuracy of the timed output itself (off the clock): the last replay's
    # prices against the oracle on a seeded sample of the batch
    accuracy = None
    if pool is not None and rank == 0 and not args.no_accuracy:
        accuracy = accuracy_sample(pool, problems, strikes, status, g_prices.cpu().numpy())
    # mixed precision: every strike of every instance against the FP64 path
    # (itself checked against the oracle), and the FP64 path's phase times
    mixed_rec = None
    if mixed and rank == 0:
        mixed_rec = mixed_vs_fp64(local_rank, batch, g_prices, status, strikes, problems, prof, args, torch,
                                  np)
    tot_s, q_all = reduce_over_ranks(sum(step_ms) / 1e3, q_ok, world, dev)
    value = q_all * args.steps / tot_s

    # end to end, as a caller pricing successive batches of this shape runs
    # it: two captured graphs in turn, so that one's read-back overlaps the
    # other's step. Every step writes the step's problem block from host
    # memory into its graph (sfft_graph_update; the replay uploads it), waits
    # for that graph's read-back of two steps before, replays it, and a copy
    # stream reads its prices and log-strikes back into pinned host memory;
    # the clock stops once the last read-back has landed. The same through
    # sfft_price_batch (host planning and uploads inside every call) is
    # e2e_direct.
    hp = [torch.empty(total_q, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    hk = [torch.empty(total_q, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    gs = [g, sfft.Graph(pricer, problems, strikes)]
    for _ in range(max(args.warmup, 1)):
        gs[1].launch()
    arr = (sfft.SfftProblem * len(problems))(*[sfft.to_c_problem(p) for p in problems])
    done = [None, None]   # event: graph j's last replay has finished
    freed = [None, None]  # event: the read-back of graph j's outputs has finished
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        j = i % 2
        main = torch.cuda.current_stream()
        if done[j] is not None:
            done[j].synchronize()  # its staging arena is free to rewrite
        gs[j]._check(gs[j].lib.sfft_graph_update(gs[j].h, arr))
        if freed[j] is not None:
            main.wait_event(freed[j])
        flush.zero_()
        gs[j].launch()
        done[j] = torch.cuda.Event()
        done[j].record(main)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(done[j])
            hp[j].copy_(gs[j].prices[:total_q], non_blocking=True)
            hk[j].copy_(gs[j].log_strikes[:total_q], non_blocking=True)
            freed[j] = torch.cuda.Event()
            freed[j].record(copy_stream)
    torch.cuda.synchronize()
    e2e_wall = time.perf_counter() - t0
    e2e_value = q_all * args.steps / e2e_wall
    for gg in gs:
        gg.close()
    dp = [prices, torch.empty_like(prices)]
    dk = [logk, torch.empty_like(logk)]
    freed = [None, None]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        j = i % 2
        main = torch.cuda.current_stream()
        if freed[j] is not None:
            main.wait_event(freed[j])
        flush.zero_()
        pricer.price_batch(batch, None, dp[j], dk[j], raise_on_error=False)
        ready = torch.cuda.Event()
        ready.record(main)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ready)
            hp[j].copy_(dp[j], non_blocking=True)
            hk[j].copy_(dk[j], non_blocking=True)
            freed[j] = torch.cuda.Event()
            freed[j].record(copy_stream)
    torch.cuda.synchronize()
    e2e_direct = q_all * args.steps / (time.perf_counter() - t0)
    h2d = args.count * (ctypes_sizeof_problem() + 20)
    d2h = 16 * total_q

    # roofline of the dominant TT kernel (FP64 ALU bound): among the phases
    # whose launches are all one kernel (a two-tier phase launches the same
    # kernel twice per step; "cross" mixes two kernels), the one with the most
    # time; achieved = its algorithmic flops over its launches' total time
    tt_phases = ["build", "zipup", "round", "readout"]
    dom = max(tt_phases, key=lambda k: prof[k]["ms"])
    dms = prof[dom]["ms"]
    achieved = prof[dom]["flops"] / (dms * 1e-3) / 1e9 if dms > 0 else 0.0
    launches = sum(v["launches"] for v in prof.values())
    traffic = None
    if (dom == "zipup" and not mixed and args.count == ZIPUP_TRAFFIC["instances"] and args.n is None
            and args.tol == 1e-12
            and kernel_src_hash() == ZIPUP_TRAFFIC["src"]):
        traffic = ZIPUP_TRAFFIC["bytes"]

    # dense-FFT baseline on the same batch: one instance per n <= 30 timed,
    # the batch time assembled from the per-n times
    dense = None
    if not args.no_dense and rank == 0:
        dense = dense_baseline(pricer, problems, strikes, torch, dev, fp64_peak)

    sweep = None
    if not args.no_config2 and rank == 0 and not mixed:
        sweep = config2_sweep(pricer, torch, dev)

    cpu = None
    if pool is not None and rank == 0 and not args.no_cpu:
        rate, one_rate, n_inst, skipped, wall, timed = oracle_sample(pool, problems, strikes,
                                                                     args.cpu_seconds, ncores)
        cpu = {"value": rate, "unit": UNIT, "cores": ncores, "kind": "oracle", "one_core_value": one_rate,
               "sample": f"{n_inst} instances of the batch in a seeded random order, each timed on "
                         f"its first max(32, 2^24/support) strikes ({timed} strikes, direct sum over "
                         f"the integrand support, {wall:.1f} s wall) and scaled to all its strikes; "
                         f"{skipped} drawn instances with support > 2^20 left out; one_core_value = "
                         f"strikes over the summed scaled seconds, value = that times the pool's "
                         f"measured concurrency"}

    phases = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                  "gflop_per_step": v["flops"] / args.steps / 1e9}
              for k, v in prof.items() if v["launches"]}
    rep_pts = float(sum(2.0 ** p.n for p, o in zip(problems, ok) if o)) * max(world, 1)
    ranks_out = [i["out_rank"] for i in info if i["status"] == 0]
    ranks_int = [i["int_rank"] for i in info if i["status"] == 0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+bf16x3 tensor-core contraction (fp32 accumulate)" if mixed else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "instances": args.count, "strikes_per_step": total_q, "priced_per_step": q_ok,
                   "failed_instances": int(len(ok) - sum(ok)), "tol": args.tol, "eta": 0.25, "alpha": 1.5,
                   "window": "|log K/S0| <= 1.5, <= 4096 strikes", "l2": "flushed (256 MB write) between steps",
                   "max_int_rank": max(ranks_int) if ranks_int else None,
                   "max_out_rank": max(ranks_out) if ranks_out else None},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "how": "successive steps of this batch shape through two captured graphs in turn "
                       "(sfft_graph_update writes each step's problem block from host memory, the "
                       "replay uploads it); each step's outputs read back to pinned host memory on a "
                       "copy stream, overlapping the other graph's step"},
        "e2e_direct": {"value": e2e_direct, "unit": UNIT,
                       "how": "the same through sfft_price_batch from the batch's host arrays, with the "
                              "host planning and uploads inside every call, outputs double-buffered"},
        "gpu_launches": launches // args.steps,
        "cold_call_ms": cold_ms,
        "roofline": {"bound": "alu", "kernel": sfft.PHASE_KERNELS[sfft.PHASE_NAMES.index(dom)],
                     "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s FP64",
                     "frac": achieved / fp64_peak if fp64_peak else None, "traffic": traffic,
                     "traffic_unit": "bytes per tier-1 launch (ncu, dram read + write)",
                     "peak_source": "measured FP64 FMA calibration (sfft_calibrate_fp64)"},
        "phases": phases,
        # secondary, as the metric's definition asks: grid points the priced
        # instances represent (sum of 2^n) per second, and FP64 work per strike
        "represented": {"value": rep_pts * args.steps / tot_s if tot_s > 0 else None,
                        "unit": "grid points/s"},
        "per_strike": {"fp64_flop": sum(v["flops"] for v in prof.values()) / args.steps / max(q_ok, 1)},
        "accuracy": accuracy,
        "mixed_precision": mixed_rec,
        "autotune": tuning,
        "direct_call": direct,
        "cpu_baseline": cpu,
        "dense_fft": dense,
        "config2_sweep": sweep,
    }
    pricer.close()
    return line


def mixed_vs_fp64(device, batch, prices, status, strikes, problems, prof, args, torch, np):
    """Price the same batch on the FP64 path (a second context, off the
    clock) and compare every strike of every instance; time the FP64 path's
    steps with the profiler for its phase times."""
    from paper_2607_28435_b300 import sfft
    ref = sfft.Pricer(device)
    try:
        p64 = torch.empty_like(prices)
        k64 = torch.empty_like(prices)
        ref.price_batch(batch, None, p64, k64, raise_on_error=False)  # warm: MPOs built
        ref.profile(True)
        ref.profile_read(reset=True)
        reps = 3
        for _ in range(reps):
            ref.price_batch(batch, None, p64, k64, raise_on_error=False)
        torch.cuda.synchronize()
        pr64 = ref.profile_read(reset=True)
        ref.profile(False)
    finally:
        ref.close()
    a, b = prices.cpu().numpy(), p64.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([s[2] for s in strikes])])
    per = np.array([np.max(np.abs(a[offs[i]:offs[i + 1]] - b[offs[i]:offs[i + 1]])) / problems[i].S0
                    if status[i] == 0 and offs[i + 1] > offs[i] else 0.0 for i in range(len(problems))])
    okm = np.array([s == 0 for s in status])
    pz = prof["zipup"]
    return {"instances": int(okm.sum()), "strikes": int(sum(s[2] for s, o in zip(strikes, okm) if o)),
            "max_abs_err_vs_fp64_over_S0": float(per.max()), "median_per_instance": float(np.median(per[okm])),
            "p99_per_instance": float(np.percentile(per[okm], 99)),
            "instances_over_1e-6": int((per > 1e-6).sum()),
            "zipup_ms_per_step": pz["ms"] / args.steps, "zipup_ms_per_step_fp64": pr64["zipup"]["ms"] / reps,
            "ms_per_step_fp64_profiled": sum(v["ms"] for v in pr64.values()) / reps,
            "tensor_core_sites_per_step": pz["evals"] / args.steps,
            "sites_per_step": float(sum(p.n for p, o in zip(problems, okm) if o)),
            "how": "every strike of every priced instance of the last timed step against the same batch on the "
                   "FP64 path (second context, off the clock); the FP64 path's times from 3 profiled steps"}


def reduce_over_ranks(seconds: float, strikes: int, world: int, device):
    """Whole-job figures across ranks: the slowest rank's time (max) and the
    strikes all ranks priced (sum). Ranks price independent instance batches,
    so this is the only cross-rank exchange (weak scaling)."""
    if world <= 1:
        return seconds, float(strikes)
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    q = torch.tensor([float(strikes)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(q, op=dist.ReduceOp.SUM)
    return float(t.item()), float(q.item())


def ctypes_sizeof_problem():
    import ctypes
    from paper_2607_28435_b300 import sfft
    return ctypes.sizeof(sfft.SfftProblem)


def config2_sweep(pricer, torch, dev, reps=3):
    """The single Heston instance of the sweep configuration (kappa 1.5768,
    theta 0.0398, sigma_v 0.5751, rho -0.5711, v0 0.0175, r 0.025, T 1, tol
    1e-12) at n = 16..40: TT-SFFT time per call (best of reps, CUDA events,
    operators cached) with the profiler's split into the integrand build and
    the core (zip-up, rounding, readout; the paper's "Core" time), and the
    dense-FFT route at n <= 32. The crossover is the smallest n from which
    the TT-SFFT call is faster than the dense one."""
    from paper_2607_28435_b300 import sfft, workloads as wl
    rows = []
    for n in range(16, 41):
        p = wl.config2_heston(n)
        st = sfft.strike_window(p)
        pr = torch.empty(max(st[2], 1), dtype=torch.float64, device=dev)
        lk = torch.empty_like(pr)
        pricer.price_batch([p], [st], pr, lk)  # builds the operator of this n
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pricer.price_batch([p], [st], pr, lk)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        pricer.profile(True)
        pricer.profile_read(reset=True)
        pricer.price_batch([p], [st], pr, lk)
        torch.cuda.synchronize()
        ph = pricer.profile_read(reset=True)
        pricer.profile(False)
        row = {"n": n, "tt_ms": best, "tt_build_ms": ph["probe"]["ms"] + ph["build"]["ms"] + ph["cross"]["ms"],
               "tt_core_ms": ph["zipup"]["ms"] + ph["round"]["ms"] + ph["readout"]["ms"], "strikes": st[2]}
        if n <= 32:
            pricer.dense_price_batch([p], [st], pr, lk)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pricer.dense_price_batch([p], [st], pr, lk)
            e1.record()
            torch.cuda.synchronize()
            row["dense_ms"] = e0.elapsed_time(e1)
        rows.append(row)
    cross = next((r["n"] for r in rows if "dense_ms" in r and r["tt_ms"] < r["dense_ms"]), None)
    core_cross = next((r["n"] for r in rows if "dense_ms" in r and r["tt_core_ms"] < r["dense_ms"]), None)
    return {"rows": rows, "crossover_n_total": cross, "crossover_n_core": core_cross,
            "how": "one Heston instance (the sweep configuration), strikes |log K/S0| <= 1.5; TT-SFFT best of "
                   f"{reps} calls with the operator cached, profiler phases from one more call; dense-FFT "
                   "route one timed call after a warm one"}


def dense_baseline(pricer, problems, strikes, torch, dev, fp64_peak):
    """The dense-FFT Carr-Madan baseline on the same batch: one instance per
    n <= 32 (SFFT_DENSE_MAX_N) timed with CUDA events, the batch time
    assembled as sum_n count_n t_n (n = 33, 34 scaled from n = 32 as
    M log M). At n = 30 and the largest n its phases are timed separately:
    the sampling of the integrand, the FFT passes, the gather."""
    by_n = {}
    for p, s in zip(problems, strikes):
        by_n.setdefault(p.n, []).append((p, s))
    t_n = {}
    phases = {}
    top_n = max(n for n in by_n if n <= 32)
    for n in sorted(by_n):
        if n > 32:
            continue
        p, s = by_n[n][0]
        pr = torch.empty(max(s[2], 1), dtype=torch.float64, device=dev)
        lk = torch.empty_like(pr)
        pricer.dense_price_batch([p], [s], pr, lk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pricer.dense_price_batch([p], [s], pr, lk)
        e1.record()
        torch.cuda.synchronize()
        t_n[n] = e0.elapsed_time(e1) / 1e3
        if n in (30, top_n):
            pricer.profile(True)
            pricer.profile_read(reset=True)
            pricer.dense_price_batch([p], [s], pr, lk)
            torch.cuda.synchronize()
            ph = pricer.profile_read(reset=True)
            pricer.profile(False)
            phases[n] = {k: ph[k]["ms"] for k in ("dense_sample", "dense_fft", "dense_gather")}
    if not t_n:
        return None
    # external reference point: cuFFT's complex-to-complex transform of the
    # same length (torch.fft on the device), FFT only, for n <= 30 (larger
    # lengths need two 32-64 GiB arrays beside the baseline's own)
    cufft = {}
    for n in sorted(t_n):
        if n > 30:
            continue
        xr = torch.zeros(1 << n, dtype=torch.complex128, device=dev)
        torch.fft.fft(xr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.fft.fft(xr)
        e1.record()
        torch.cuda.synchronize()
        cufft[str(n)] = e0.elapsed_time(e1) / 1e3
        del xr
    top = max(t_n)
    est = 0.0
    extrapolated = []
    for n, items in by_n.items():
        if n in t_n:
            est += len(items) * t_n[n]
        else:
            est += len(items) * t_n[top] * 2.0 ** (n - top) * n / top
            extrapolated.append(n)
    q = sum(s[2] for s in strikes)
    out = {"value": q / est, "unit": UNIT, "batch_seconds": est, "measured_n": sorted(t_n),
           "seconds_per_n": {str(k): v for k, v in sorted(t_n.items())},
           "extrapolated_n": sorted(extrapolated),
           "cufft_z2z_seconds_per_n": cufft,
           "how": "one instance per n timed (CUDA events); batch time = sum_n count_n t_n; n > 32 scaled as "
                  "M log M from n = 32; phases at n = 30 and the largest n from the profiler; cuFFT (torch.fft) of the "
                  "same lengths up to n = 30 as an external reference"}
    for n, ph in sorted(phases.items()):
        m, npass = 1 << n, (n + 9) // 10  # passes of at most 2^10-point sub-transforms
        fft_ms = ph["dense_fft"]
        rec = dict(ph)
        if fft_ms:
            # every pass reads and writes 16 M bytes; the FFT work is 5 M log2 M
            rec["fft_passes"] = npass
            rec["fft_passes_hbm_gbs"] = 32.0 * m * npass / (fft_ms * 1e-3) / 1e9
            if fp64_peak:
                rec["fft_passes_fp64_frac"] = 5.0 * m * n / (fft_ms * 1e-3) / 1e9 / fp64_peak
        if str(n) in cufft:
            # our FFT passes against cuFFT's Z2Z of the same length
            rec["cufft_z2z_ms"] = cufft[str(n)] * 1e3
            rec["fft_over_cufft"] = fft_ms / (cufft[str(n)] * 1e3) if fft_ms else None
        out.setdefault("phases_ms", {})[str(n)] = rec
    return out


# --------------------------------------------------------------------------- reference arm
def run_reference(args, pool, ncores):
    from paper_2607_28435_b300 import workloads as wl
    from oracle import carr_madan as cm
    problems = batch_problems(args)
    strikes = [cm.strike_window(p) for p in problems]
    rates = []
    for i in range(args.warmup + args.steps):
        rate, _, n_inst, skipped, wall, timed = oracle_sample(pool, problems, strikes,
                                                              args.cpu_seconds, ncores)
        if i >= args.warmup:
            rates.append(rate)
    value = statistics.mean(rates)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(args)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"per step, {n_inst} instances in a seeded random order, each timed on "
                                   f"its first max(32, 2^24/support) strikes and scaled to all its strikes "
                                   f"(direct sum over the support); {skipped} drawn instances with support "
                                   f"> 2^20 left out"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    ncores = len(os.sched_getaffinity(0))
    pool = None
    if rank == 0 and (args.impl == "reference" or not args.no_cpu or not args.no_accuracy):
        pool = oracle_pool(ncores)
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, pool, ncores)), flush=True)
        if pool:
            pool.close()
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group(backend="nccl")
    line = run_ours(args, rank, world, local_rank, pool, ncores)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pool:
        pool.close()
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
