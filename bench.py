"""Benchmark: window updates/s of the sliding-window cumulant path on GB300.

One step = one window shift of the whole hot path: ring append / X_(-)
extraction, moment-sum update of orders 1..d, moment-to-cumulant recovery of
orders 1..d, and the norm reduction (Algorithm 1, one loop iteration).

Default workload: n=48 variables, orders 1..6, block size 4, window T=2^16,
shift p=2^12, FP32 samples from a multivariate t(5) with a random correlation
matrix, seeded and synthetic: the largest single-window configuration, whose
order-6 moment tensor (50.7 M stored elements, 405 MB in FP64) is larger than
L2.  The plain FP64 form is measured on the same stream beside the mixed one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|bf16|fp16]
    python bench.py --impl reference      # the CPU oracle on the same workload
    python bench.py --workload n32_d4_b4_T4096_ica --grad   # forward + backward

Prints one JSON line (rank 0).  Under torchrun each rank advances its own
independent stream (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import functools
import itertools
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1701_06446_gb300 import ranks  # noqa: E402
from paper_1701_06446_gb300.streams import WORKLOADS  # noqa: E402

METRIC = "window updates/s and TFLOP/s vs tensor-core peak at stated error vs FP64 oracle"
UNIT = "window updates/s"
DEFAULT_WORKLOAD = "n48_d6_b4_T65536_p4096"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2
FP32_LANES_PER_SM = 128     # FP32 FMA-pipe lanes per SM (Blackwell)
TWO_WORD_MIN_ORDER = 5      # orders whose subset products run in two-word FP32 arithmetic
TWO_WORD_OPS_PER_TERM = 12  # FP32 operations of one two-word multiply-accumulate


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# drift limit of the library's automatic re-centring in the mixed forms (standard deviations)
AUTO_RECENTER = 0.25


def canonical_order(b: int, s: int) -> bool:
    """Orders the library recovers per canonical element (single windows)."""
    return 5 <= s <= 6 and b ** s >= 256 and b ** (s - 1) <= 0xffff


def _run_mask_count(j, b):
    """In-block offsets of the sorted block tuple j whose digits do not decrease
    inside its runs of equal entries: prod over runs of C(b + r - 1, r)."""
    cnt, i = 1, 0
    while i < len(j):
        r = i
        while r + 1 < len(j) and j[r + 1] == j[i]:
            r += 1
        cnt *= math.comb(b + r - i, r - i + 1)
        i = r + 1
    return cnt


@functools.lru_cache(maxsize=None)
def gemm_outputs(n: int, b: int, s: int) -> int:
    """Outputs of the order-s update GEMM: E_s, or, for a canonical order,
    (rows canonical in the left tuple) x (columns canonical in the right tuple)
    summed over the pairs that form sorted blocks."""
    from paper_1701_06446_gb300 import layout_size
    if not canonical_order(b, s):
        return layout_size(n, b, s)
    nb = -(-n // b)
    h = (s + 1) // 2
    left = list(itertools.combinations_with_replacement(range(nb), h))
    right = list(itertools.combinations_with_replacement(range(nb), s - h))
    rows = [0] * nb
    for jl in left:
        rows[jl[-1]] += _run_mask_count(jl, b)
    cols = [0] * (nb + 1)  # columns of the right tuples whose first block is >= m
    for jr in right:
        cols[jr[0]] += _run_mask_count(jr, b)
    for m in range(nb - 1, -1, -1):
        cols[m] += cols[m + 1]
    return sum(rows[m] * cols[m] for m in range(nb))


@functools.lru_cache(maxsize=None)
def operand_rows(n: int, b: int, d: int) -> int:
    """Distinct Khatri-Rao operand rows the update builds per shift: for every order
    a left factor of ceil(s/2) variables (rows grouped by their last block) and a
    right factor of the rest (lexicographic), a set of each (factor count,
    grouping, compression) built once and shared between orders; compressed sets
    (canonical orders) keep the digit rows that do not decrease inside a tuple's
    runs of equal blocks."""
    nb = -(-n // b)
    sets = set()
    for s in range(1, d + 1):
        h = (s + 1) // 2
        comp = canonical_order(b, s)
        for k, grouped in ((h, 1), (s - h, 0)):
            sets.add((k, grouped if k > 1 else 0, comp if k > 1 else False))
    rows = 0
    for k, _, comp in sets:
        if k == 0:
            rows += 1
            continue
        for j in itertools.combinations_with_replacement(range(nb), k):
            rows += _run_mask_count(j, b) if comp else b ** k
    return rows


def algorithmic_work(W, fifo: bool = False) -> dict:
    """Algorithmic work of one shift.

    * update: 2 * K flops (one product per multiply-add) per element the recovery
      needs, K = 2p samples (entering and leaving), or K = p when the leaving
      batch's sums come from the batch-sum FIFO.  Orders with the canonical
      recovery need their canonical elements only (one per class of entries that
      super-symmetry makes equal; the other stored elements of a diagonal block are
      copies), the others every stored element E_s.  `update_issued`: the products
      the update actually forms (`gemm_outputs`: the compressed update tables of
      the canonical orders also produce the elements that are canonical in each
      half but not across the junction); the tensor pipe issues three MMAs per
      product in the split forms (hi*hi + hi*lo + lo*hi).
    * recovery, per element of order s: 2^{s-1} - 1 subset terms.  Orders 5-6 with
      blocks of >= 256 elements are recovered once per class of entries that
      super-symmetry makes equal (C(n_pad + s - 1, s) canonical elements instead of
      E_s stored ones; the copies are memory traffic), the others per stored element.  Orders
      below TWO_WORD_MIN_ORDER run them as FP64 multiply-adds, plus the 1/T
      scaling, the multiplicity-weighted square (2) and the fold of the shift's
      batch sums (2): `recovery_fp64` flops.  Orders from TWO_WORD_MIN_ORDER up (mixed
      forms) run each term as a two-word FP32 multiply-accumulate
      (TWO_WORD_OPS_PER_TERM FP32 operations on the FMA pipe): `recovery_fp32_ops`.
    * recovery bytes, per element whose sums are kept (every stored element, or the
      canonical elements of the canonical orders): the FP64 sum read and written
      (16), the shift's FP32 tile sum read (4) and the FIFO slot read and written
      (8, FIFO) or the leaving tile sum read (4); the cumulant written at every
      stored element (8); orders below d also write their two-word copies (16) in
      the forms that have them, at the canonical elements only for canonical orders
      (the orders above read no others).
    """
    from paper_1701_06446_gb300 import layout_size
    E = {s: layout_size(W.n, W.b, s) for s in range(1, W.d + 1)}
    K = W.p if fifo else 2 * W.p
    terms = {s: 2 ** (s - 1) - 1 for s in E}
    two_word = W.d >= TWO_WORD_MIN_ORDER
    fp64 = sum((2.0 * terms[s] + 5.0) * E[s] for s in E if not (two_word and s >= TWO_WORD_MIN_ORDER))
    npad = -(-W.n // W.b) * W.b
    Ecomp = {s: math.comb(npad + s - 1, s) if canonical_order(W.b, s) else E[s] for s in E}
    upd = sum(2.0 * K * Ecomp[s] for s in E)
    upd_issued = sum(2.0 * K * gemm_outputs(W.n, W.b, s) for s in E)
    fp32_ops = sum(TWO_WORD_OPS_PER_TERM * terms[s] * Ecomp[s] for s in E if two_word and s >= TWO_WORD_MIN_ORDER)
    per_kept = 16 + 4 + (8 if fifo else 4)
    rec_bytes = sum(per_kept * Ecomp[s] + 8 * E[s] + (16 * Ecomp[s] if two_word and s < W.d else 0) for s in E)
    npad_ = -(-W.n // W.b) * W.b
    # operand build: hi and lo 16-bit words of every row for each staged sample written,
    # the staged FP32 samples read
    build_bytes = operand_rows(W.n, W.b, W.d) * K * 2 * 2 + npad_ * K * 4
    return {"update": upd, "update_issued": upd_issued, "build_bytes": build_bytes,
            "recovery_fp64": fp64, "recovery_fp32_ops": fp32_ops,
            "recovery_bytes": rec_bytes, "elements": E, "computed_elements": Ecomp, "two_word": two_word}


# DRAM bytes (read + write) per shift from an ncu capture of the current kernels (profiles/
# launches_*.md), by workload: the recovery's launches of one shift, the GEMM, and the staging
# plus operand build.  The n=48 workload's were taken with a window of 2^13 samples, whose
# per-launch work is the same.  None where no capture of the current kernels exists.
RECOVERY_TRAFFIC: dict[str, int] = {"n60_d4_b3_T32768_p1024": 13007616}
GEMM_TRAFFIC: dict[str, int] = {"n48_d6_b4_T65536_p4096": 1508085230, "n60_d4_b3_T32768_p1024": 15829120}
BUILD_TRAFFIC: dict[str, int] = {"n48_d6_b4_T65536_p4096": 641766161}


def fp64_peak_tflops(dev) -> float:
    """Measured FP64 rate of this GPU: cuBLAS DGEMM 4096^3 through torch, best of 3
    (CUDA events), as the bf16 peak of MEASURED_PEAKS.json is a cuBLAS GEMM."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del a, b
    return 2.0 * 4096 ** 3 / best / 1e12


def device_uuid(dev):
    """nvidia-smi's id of the torch device (its UUID), or None."""
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if device_id:
            cmd += ["-i", device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the --impl reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(X: np.ndarray, W, per_order: int, seed: int, full_upto: int) -> tuple[float, float, str]:
    """Time the oracle on a bounded sample of one full recomputation of C_1..C_d for
    window X: every sorted tuple of the orders <= full_upto, `per_order` seeded sorted
    tuples of each higher order.  Returns (seconds measured, seconds the whole
    recomputation would take -- the sampled orders extrapolated linearly by tuple
    count --, a description)."""
    import itertools

    import oracle
    t0 = time.perf_counter()
    cen = oracle.center(X)
    measured = time.perf_counter() - t0
    total = measured
    parts = []
    for s in range(1, W.d + 1):
        n_tuples = math.comb(W.n + s - 1, s)
        if s <= full_upto or n_tuples <= per_order:
            tup = np.array(list(itertools.combinations_with_replacement(range(W.n), s)), np.int32)
            t0 = time.perf_counter()
            oracle.cumulant_tuples(X, tup, centred=cen)
            dt = time.perf_counter() - t0
            measured += dt
            total += dt
            parts.append(f"order {s}: all {n_tuples} tuples")
        else:
            tup = oracle.sample_sorted_tuples(W.n, s, per_order, seed + s)
            t0 = time.perf_counter()
            oracle.cumulant_tuples(X, tup, centred=cen)
            dt = time.perf_counter() - t0
            measured += dt
            total += dt * n_tuples / per_order
            parts.append(f"order {s}: {per_order} of {n_tuples} tuples (extrapolated)")
    return measured, total, "; ".join(parts)


def oracle_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, W, rank: int):
    """The oracle as the reference arm, on the machine's host cores (rank 0 only).
    Each step is one timed bounded sample of a full-window recomputation (all
    tuples of orders <= 2, `--ref-tuples` seeded tuples of each higher order, a
    different seed per step): `ms_per_step` is that sample's measured time, and
    `value` (window updates/s) is 1 / the full recomputation time extrapolated
    from the samples, stated as such."""
    if rank != 0:
        return
    X = W.stream().rows(0, W.T).astype(np.float64)
    for k in range(args.warmup):
        oracle_sample(X, W, max(1, args.ref_tuples // 10), seed=100 + k, full_upto=1)
    measured, total = [], []
    sample = ""
    t_start = time.perf_counter()
    for k in range(args.steps):
        m, t, sample = oracle_sample(X, W, args.ref_tuples, seed=k, full_upto=2)
        measured.append(m)
        total.append(t)
    wall = time.perf_counter() - t_start
    per_window = statistics.mean(total)
    value = 1.0 / per_window
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(W, "fp64-oracle"),
        "sample_s_per_step": statistics.mean(measured),
        "extrapolated_s_per_window": per_window,
        "value_basis": "1 / full-window recomputation time extrapolated by tuple count from the timed samples",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": f"per step, one bounded sample of a full recomputation: {sample}; "
                                   f"measured {statistics.mean(measured):.3f} s per step, "
                                   f"extrapolated {per_window:.4g} s per window"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(W, precision: str) -> dict:
    return {"workload": W.name, "n": W.n, "orders": f"1..{W.d}", "b": W.b, "T": W.T, "p": W.p,
            "precision": precision, "stream": W.kind,
            "l2": "flushed (256 MB write) between timed steps"}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def sampled_error(h, X: np.ndarray, per_order: int = 200) -> dict:
    import oracle
    cen = oracle.center(X)
    out = {}
    for s in range(1, h.d + 1):
        C = h.cumulants(s).cpu().numpy()
        tup = oracle.sample_sorted_tuples(h.n, s, per_order, seed=1000 + s)
        idx = np.array([oracle.storage_index(h.n, h.b, t) for t in tup])
        ref = oracle.cumulant_tuples(X, tup, centred=cen)
        out[str(s)] = float(np.linalg.norm(C[idx] - ref) / max(np.linalg.norm(ref), 1e-300))
    return out


def measure_fp64_form(W, stream, base: int, steps: int, dev) -> dict:
    """The plain FP64 GPU form on the same stretch of the stream, for comparison
    (FP64 products and sums, the paper's arithmetic): window updates/s with the
    L2 flushed before every timed shift, and its update's FP64 rate."""
    import torch
    from paper_1701_06446_gb300 import CumWin
    X = torch.from_numpy(stream.rows(base, base + W.T + (steps + 3) * W.p)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    h = CumWin(W.n, W.d, W.b, W.T, W.p, "fp64", device=dev)
    h.fill(X[: W.T])
    for k in range(3):
        h.push(X[W.T + k * W.p: W.T + (k + 1) * W.p])
    torch.cuda.synchronize()
    h.set_timing(True)
    st = torch.cuda.current_stream(dev)
    total = 0.0
    for k in range(3, 3 + steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h.push(X[W.T + k * W.p: W.T + (k + 1) * W.p])
        e1.record(st)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    t = h.get_timing()
    fifo = bool(h.fifo)  # regular shifts subtract the leaving batch's stored FP64 sums
    h.close()
    ms = total / steps
    upd = t["update_ms"] / max(t["shifts"], 1)
    work = algorithmic_work(W, fifo)
    return {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "update_ms": upd,
            "update_tflops": work["update"] / (upd * 1e-3) / 1e12,
            "update_issued_tflops": work["update_issued"] / (upd * 1e-3) / 1e12, "steps": steps,
            "fifo": fifo, "l2": "flushed before every timed shift"}


# per-order relative Frobenius bounds of the final window against the oracle, about 3x the
# error measured on GB300, per workload and form
ERROR_BOUND = {
    "n48_d6_b4_T65536_p4096": {"bf16": {1: 3e-5, 2: 6e-5, 3: 5e-5, 4: 4e-5, 5: 3e-5, 6: 3e-5},
                               "fp16": {1: 3e-5, 2: 7e-5, 3: 4e-5, 4: 3e-5, 5: 2e-5, 6: 2e-5}},
    "n60_d4_b3_T32768_p1024": {"bf16": {1: 2e-5, 2: 2e-5, 3: 2e-5, 4: 2e-4},
                               "fp16": {1: 2e-5, 2: 2e-5, 3: 2e-5, 4: 2e-4}},
}


def run_ours(args, W, rank: int, world: int):
    import torch
    from paper_1701_06446_gb300 import CumWin

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    precision = args.precision
    stream = W.stream()
    split_steps = min(args.steps, 50)  # the instrumented pass after the timed region
    nsteps = args.warmup + args.steps + split_steps
    e2e_steps = min(args.steps, 200)
    # each rank advances its own independent stretch of the stream
    e2e_reps = 3  # streaming loops over fresh stretches of the stream; the median is reported
    base = ranks.stream_base(rank, W.T, W.p, nsteps + (e2e_reps + 1) * e2e_steps)
    ksplit = None
    X = stream.rows(base, base + W.T + nsteps * W.p)
    Xd = torch.from_numpy(X).to(dev)
    h = CumWin(W.n, W.d, W.b, W.T, W.p, precision, device=dev)
    if precision != "fp64":  # the library's drift policy (a user of a drifting stream turns it on)
        h.set_auto_recenter(AUTO_RECENTER)
    h.fill(Xd[: W.T])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    batches = [Xd[W.T + k * W.p: W.T + (k + 1) * W.p] for k in range(nsteps)]
    for k in range(args.warmup):
        h.push(batches[k])
        if k == 0 and precision != "fp64":
            ksplit = h.tune(20)  # untimed: pick the tensor-core K-split on real data
    torch.cuda.synchronize()

    st = torch.cuda.current_stream(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ranks.barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(device_uuid(dev)) if rank == 0 else None
    # coarse library timing inside the timed region: the recovery's own interval (the
    # dominant kernel) without an event between the operand build and the GEMM
    h.set_timing(2)
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(st)
        h.push(batches[args.warmup + k])
        ends[k].record(st)
    torch.cuda.synchronize()
    ranks.barrier(world)
    clocks = sampler.stop() if sampler else None
    timing = h.get_timing()
    h.set_timing(False)
    # the staging / GEMM split from an untimed pass with every phase event (the next shifts
    # of the stream, L2 flushed before each)
    h.set_timing(True)
    for k in range(split_steps):
        flush.zero_()
        h.push(batches[args.warmup + args.steps + k])
    timing_split = h.get_timing()
    h.set_timing(False)
    step_ms = ranks.max_over_ranks([sum(s.elapsed_time(e) for s, e in zip(starts, ends))], dev, world)[0]
    ms_per_step = step_ms / args.steps
    value = ranks.job_rate(world, args.steps, step_ms * 1e-3)
    del batches, Xd

    # end-to-end through the C ABI with host buffers: H2D of X_(+) from pinned memory and D2H of
    # every step's ||C_s||, nu_s and status inside the timed region.  Streaming form: each push's
    # estimators are formed on the device and enqueued behind its recovery (which overlaps the
    # next push); one synchronisation at the end.  Synchronous form: norms() blocks after every push.
    e2e_steps_total = (e2e_reps + 1) * e2e_steps
    host = torch.from_numpy(stream.rows(base + W.T + nsteps * W.p,
                                        base + W.T + (nsteps + e2e_steps_total) * W.p)).pin_memory()
    hb = [host[k * W.p:(k + 1) * W.p] for k in range(e2e_steps_total)]
    fro_host = torch.zeros(e2e_steps, W.d, dtype=torch.float64).pin_memory()
    nu_host = torch.zeros(e2e_steps, W.d, dtype=torch.float64).pin_memory()
    st_host = torch.full((e2e_steps,), -1, dtype=torch.int32).pin_memory()
    stream_s = []
    for r in range(e2e_reps):
        st_host.fill_(-1)
        torch.cuda.synchronize()
        ranks.barrier(world)
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            h.push_host(hb[r * e2e_steps + k])
            h.estimators_enqueue(fro_host[k], nu_host[k], st_host[k:k + 1])
        h.join()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if int(st_host.abs().max()) != 0:
            raise RuntimeError("device status reported an error during the end-to-end loop")
        stream_s.append(ranks.max_over_ranks([t1 - t0], dev, world)[0])
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for k in range(e2e_reps * e2e_steps, e2e_steps_total):
        h.push_host(hb[k])
        fro, nu = h.norms()
    t3 = time.perf_counter()
    e2e_value = ranks.job_rate(world, e2e_steps, statistics.median(stream_s))
    e2e_sync_value = ranks.job_rate(world, e2e_steps, ranks.max_over_ranks([t3 - t2], dev, world)[0])

    # accuracy of the final window against the FP64 oracle (sampled tuples)
    final = stream.rows(base + (nsteps + e2e_steps_total) * W.p, base + W.T + (nsteps + e2e_steps_total) * W.p)
    err = sampled_error(h, final) if rank == 0 else None

    if rank != 0:
        h.close()
        return
    fifo = bool(h.fifo)
    tiles = h.tiles()
    recenter = None
    if precision != "fp64":
        r_, k_ = h.drift()
        recenter = {"limit": AUTO_RECENTER, "recenters": k_, "last_drift": r_,
                    "note": "re-centre (recompute the window's sums about its column means) when the mean "
                            "drifts more than `limit` standard deviations from the shift; its cost is inside "
                            "whichever loop it falls in"}
    work = algorithmic_work(W, fifo)
    peaks, peak_kind = _peaks()
    # the timed region's events: the update (staging, operand build, GEMM) and the recovery;
    # the instrumented pass adds an event between the operand build and the GEMM, which
    # gives the staging + build time.  (Its interval from that event to the GEMM's end
    # comes out about 0.2 ms shorter than the GEMM's own duration at n=48, and the update
    # of the instrumented pass shorter than the timed region's by as much, so the GEMM's
    # time is taken as the timed update minus the staging + build.)
    rec_ms = timing["cumulant_ms"] / max(timing["shifts"], 1)
    upd_ms = timing["update_ms"] / max(timing["shifts"], 1)
    stg_ms = timing_split["stage_ms"] / max(timing_split["shifts"], 1)
    h.close()
    fp64_peak = fp64_peak_tflops(dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = sm_count * FP32_LANES_PER_SM * clk_mhz * 1e6 / 1e12  # T FP32 lane ops/s
    rec_s = rec_ms * 1e-3
    if W.d <= 4:
        rec_names = "k_recover_fused"
    else:
        hi = [f"k_canon<{s_}> + k_canon_expand" if canonical_order(W.b, s_) else f"k_cumulants<{s_}>"
              for s_ in range(5, W.d + 1)]
        rec_names = "recovery: k_recover_fused<4>, k_split, " + ", ".join(hi) + ", k_norm_final"
    rec_common = {"kernel": rec_names, "avg_launch_ms": rec_ms, "share_of_step": rec_ms / ms_per_step,
                  "traffic": RECOVERY_TRAFFIC.get(W.name)}
    if precision == "fp64":
        achieved = work["update"] / (upd_ms * 1e-3) / 1e12
        roof = {"kernel": "k_update_f64", "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "peak_kind": "measured FP64 (cuBLAS DGEMM 4096^3 in this run)", "traffic": None,
                "per_launch": f"{work['update']:.4g} algorithmic flops (2 x 2p per element the recovery "
                              f"needs: canonical elements of the canonical orders, E_s of the others; "
                              f"{work['update_issued']:.4g} formed by the compressed update tables)",
                "avg_launch_ms": upd_ms}
        roof_other = None
        roof_hbm = None
        roof_build = None
    else:
        # the GEMM alone: the update phase minus the staging and operand build before it
        gemm_ms = max(upd_ms - stg_ms, 1e-6)
        achieved = work["update"] / (gemm_ms * 1e-3) / 1e12
        # a launch of well under a millisecond per shift: the burst figure (the sustained
        # one is a seconds-long loop that the power cap held near 1.5 GHz)
        peak = peaks.get("bf16_tflops", 1900.0)
        roof_gemm = {"kernel": "k_kr_gemm", "bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "issued_frac": 3.0 * work["update_issued"] / (gemm_ms * 1e-3) / 1e12 / peak,
                     "peak_kind": f"{peak_kind} bf16 burst (of {peak_kind})",
                     "traffic": GEMM_TRAFFIC.get(W.name), "avg_launch_ms": gemm_ms,
                     "share_of_step": gemm_ms / ms_per_step,
                     "per_launch": f"{work['update']:.4g} algorithmic flops (2 x K per element the recovery "
                                   f"needs, K = {'p: entering samples; leaving sums from the FIFO' if fifo else '2p'}: "
                                   f"the canonical elements of the canonical orders, E_s of the others); the GEMM "
                                   f"forms {work['update_issued']:.4g} (compressed update tables) and the tensor "
                                   f"pipe issues 3x those (hi*hi + hi*lo + lo*hi): issued_frac"}
        if work["two_word"]:
            # the recovery's time goes to the two-word products of the orders >= 5 on the FMA pipe
            ops = work["recovery_fp32_ops"] / rec_s / 1e12
            roof_rec = dict(rec_common, bound="alu", achieved=ops, peak=fp32_peak, unit="Tops/s",
                            frac=ops / fp32_peak,
                            peak_kind=f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                      f"{clk_mhz:.0f} MHz (median SM clock of the timed region)",
                            per_launch=f"{work['recovery_fp32_ops']:.4g} FP32 operations: per computed element "
                                       f"(canonical: one per class of equal entries) of order s >= "
                                       f"{TWO_WORD_MIN_ORDER}, 2^(s-1)-1 subset terms x "
                                       f"{TWO_WORD_OPS_PER_TERM} (two-word multiply-accumulate); the orders "
                                       f"below run on the FP64 pipe ({work['recovery_fp64']:.3g} flops)")
        else:
            fl = work["recovery_fp64"] / rec_s / 1e12
            roof_rec = dict(rec_common, bound="alu", achieved=fl, peak=fp64_peak, unit="TFLOP/s",
                            frac=fl / fp64_peak,
                            peak_kind="measured FP64 (cuBLAS DGEMM 4096^3 in this run)",
                            per_launch=f"{work['recovery_fp64']:.4g} algorithmic FP64 flops (per stored element "
                                       f"of order s: 2(2^(s-1)-1) subset recursion + 1 scaling + 2 norm + 2 fold)")
        gbs = work["recovery_bytes"] / rec_s / 1e9
        roof_hbm = dict(rec_common, bound="hbm", achieved=gbs, peak=peaks["hbm_gbs"], unit="GB/s",
                        frac=gbs / peaks["hbm_gbs"], peak_kind=f"{peak_kind} HBM copy (of {peak_kind})",
                        per_launch=f"{work['recovery_bytes']:.4g} algorithmic bytes (per element whose sums "
                                   f"are kept, the canonical ones of the canonical orders: FP64 sum read + write, "
                                   f"FP32 tile sum read, FIFO slot read + write, two-word copies of the orders "
                                   f"below d; per stored element: the cumulant write)")
        bgbs = work["build_bytes"] / (stg_ms * 1e-3) / 1e9
        roof_build = {"kernel": "k_tc_stage_push + k_kr_build", "bound": "hbm", "achieved": bgbs,
                      "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": bgbs / peaks["hbm_gbs"],
                      "peak_kind": f"{peak_kind} HBM copy (of {peak_kind})",
                      "traffic": BUILD_TRAFFIC.get(W.name) if precision == "bf16" else None,
                      "avg_launch_ms": stg_ms, "share_of_step": stg_ms / ms_per_step,
                      "per_launch": f"{work['build_bytes']:.4g} algorithmic bytes: {operand_rows(W.n, W.b, W.d)} "
                                    f"operand rows x {W.p if fifo else 2 * W.p} samples x hi + lo 16-bit "
                                    f"words written, the staged FP32 samples read"}
        # the roofline line is the dominant kernel's; the other is kept beside it
        if rec_ms >= gemm_ms:
            roof, roof_other = roof_rec, roof_gemm
        else:
            roof, roof_other = roof_gemm, roof_rec
    cpu = None
    fp64_form = None
    if precision != "fp64" and args.fp64_steps > 0:
        fp64_form = measure_fp64_form(W, stream, base, args.fp64_steps, dev)
        fp64_form["update_frac_of_fp64_peak"] = fp64_form["update_tflops"] / fp64_peak
        fp64_form["update_issued_frac_of_fp64_peak"] = fp64_form["update_issued_tflops"] / fp64_peak
    if world == 1 and not args.no_cpu_baseline:
        Xw = final.astype(np.float64)
        m, tot, sample = oracle_sample(Xw, W, args.cpu_tuples, seed=7, full_upto=3)
        cpu = {"value": 1.0 / tot, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": f"one full recomputation of the final window: {sample}; measured {m:.2f} s, "
                         f"extrapolated {tot:.4g} s per window",
               "sample_s": m, "extrapolated_s_per_window": tot}
    bound = {s_: 1e-10 for s_ in range(1, 9)} if precision == "fp64" else \
        ERROR_BOUND.get(W.name, {}).get(precision, {})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == "fp64" else f"{precision}x3+f32acc+f64sum",
        "data": "synthetic", "config": dict(config_of(W, precision), ksplit=ksplit, fifo=fifo, tiles=tiles,
                                            auto_recenter=recenter),
        "samples_per_s": value * W.p,
        "tflops": work["update"] / (ms_per_step * 1e-3) / 1e12,
        "stage_ms": stg_ms, "update_ms": upd_ms, "recovery_ms": rec_ms,
        "fp64_form": fp64_form,
        "error_vs_oracle": {"metric": "relative Frobenius error per order on 200 sampled tuples",
                            "per_order": err,
                            "bound": {str(s_): bound.get(s_) for s_ in range(1, W.d + 1)},
                            "within_bound": (all(err[str(s_)] <= bound[s_] for s_ in range(1, W.d + 1))
                                             if err and len(bound) >= W.d else None)},
        "roofline": roof, "roofline_other": roof_other, "roofline_recovery_hbm": roof_hbm,
        "roofline_build": roof_build,
        "fp64_peak_tflops_measured": fp64_peak, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": W.p * W.n * 4,
                "d2h_bytes_per_step": 2 * W.d * 8 + 4, "steps": e2e_steps, "loops": e2e_reps,
                "form": "push_host + estimators_enqueue per step (||C_s||, nu_s and status formed on the device "
                        "and copied to pinned host memory behind the pipelined recovery), one synchronisation at "
                        "the end of each loop; no L2 flush; median of the loops",
                "synchronous": {"value": e2e_sync_value, "unit": UNIT,
                                "form": "push_host + blocking norms() per step"}},
        "gpu_launches": timing["launches"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_grad(args, W, rank: int, world: int):
    """Forward + backward of L = sum_s w_s ||C_s||_F^2 (w_3 = w_4 = 1) for the T x n
    window of the ICA workload: the window is loaded as a fresh window (all moments
    recomputed), L formed on the device, and dL/dX computed by the adjoint, per step."""
    import torch
    from paper_1701_06446_gb300 import CumWin

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(5 + rank)
    X0 = W.stream().rows(0, W.T)
    # each step a different window: the source rows permuted (same distribution)
    Xs = [torch.from_numpy(np.ascontiguousarray(X0[rng.permutation(W.T)])).to(dev)
          for _ in range(args.warmup + args.steps)]
    w = [0.0, 0.0, 0.0, 1.0, 1.0][: W.d + 1]
    h = CumWin(W.n, W.d, W.b, W.T, W.p, "fp64", device=dev)
    L = torch.empty((), dtype=torch.float64, device=dev)
    for k in range(args.warmup):
        h.fill(Xs[k])
        h.loss(w, L)
        h.grad(w)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream(dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    fwd = bwd = 0.0
    ranks.barrier(world)
    sampler = ClockSampler(device_uuid(dev)) if rank == 0 else None
    for k in range(args.steps):
        e0.record(st)
        h.fill(Xs[args.warmup + k])
        h.loss(w, L)
        e1.record(st)
        g = h.grad(w)
        e2.record(st)
        torch.cuda.synchronize()
        fwd += e0.elapsed_time(e1)
        bwd += e1.elapsed_time(e2)
    clocks = sampler.stop() if sampler else None
    ms = ranks.max_over_ranks([(fwd + bwd) / args.steps], dev, world)[0]
    # error against the oracle's closed-form gradient on the last window
    import oracle
    ref = oracle.grad(Xs[-1].cpu().numpy().astype(np.float64), w)
    gerr = float(np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref))
    h.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": ranks.job_rate(world, 1, ms * 1e-3), "unit": "forward+backward passes/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 sums, f32 adjoint",
            "data": "synthetic", "config": dict(config_of(W, "fp64"), loss="w3 = w4 = 1",
                                                 l2="window and state smaller than L2, no flush"),
            "forward_ms": fwd / args.steps, "backward_ms": bwd / args.steps,
            "grad_rel_error_vs_oracle": gerr, "clocks": clocks}
    print(json.dumps(line), flush=True)


BATCH_WORKLOAD = "batch512_b4_p256"


def run_batch(args, rank: int, world: int):
    """512 independent windows (n in 8..64, d in {3,4}, T in {2^12, 2^14},
    Gaussian or t(4), b=4, p=256), all advanced by one captured CUDA graph per
    shift.  Reports window updates/s over all windows and the per-shift
    latency (p50/p99 over >= 1000 graph replays)."""
    import torch
    from paper_1701_06446_gb300 import CumWinBatch
    from paper_1701_06446_gb300.streams import Stream, batched_streams

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    params = batched_streams(seed=4 + 1000 * rank, count=512)
    b, p = 4, 256
    ns, ds, Ts = [q["n"] for q in params], [q["d"] for q in params], [q["T"] for q in params]
    streams = [Stream(q["kind"], q["n"], q["seed"]) for q in params]
    nsteps = args.warmup + min(args.steps, 64)
    ksplit = None
    t_gen = time.perf_counter()
    firsts = [torch.from_numpy(st.rows(0, T)).to(dev) for st, T in zip(streams, Ts)]
    cap_stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(cap_stream):
        B = CumWinBatch(ns, ds, Ts, b, p, args.precision, device=dev)
        packs = [B.pack([torch.from_numpy(st.rows(T + k * p, T + (k + 1) * p)).to(dev)
                         for st, T in zip(streams, Ts)]) for k in range(nsteps)]
        B.fill(firsts)
        buf = packs[0].clone()
        for k in range(args.warmup):
            B.push(packs[k])
            if k == 0:
                ksplit = B.tune(20)  # untimed: pick the tensor-core K-split on real data
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(g, stream=cap_stream):
            B.push(buf)
    torch.cuda.synchronize()
    steps = nsteps - args.warmup
    st0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    st1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches_per_shift = B.launches()  # the eager push before the capture launched the same kernels
    ranks.barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(device_uuid(dev)) if rank == 0 else None
    with torch.cuda.stream(cap_stream):
        for k in range(steps):
            buf.copy_(packs[args.warmup + k])
            st0[k].record(cap_stream)
            g.replay()
            st1[k].record(cap_stream)
    torch.cuda.synchronize()
    ranks.barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = [a.elapsed_time(z) for a, z in zip(st0, st1)]
    # latency over >= 1000 replays (inputs cycle through the same packs)
    reps = max(1000, steps)
    l0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    l1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    with torch.cuda.stream(cap_stream):
        for k in range(reps):
            buf.copy_(packs[k % nsteps])
            l0[k].record(cap_stream)
            g.replay()
            l1[k].record(cap_stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(z) for a, z in zip(l0, l1))
    # the same shifts phase by phase (separate launches, one graph per shift), for comparison
    phased = None
    if B.set_single_launch(False):
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap_stream):
            with torch.cuda.graph(g2, stream=cap_stream):
                B.push(buf)
        torch.cuda.synchronize()
        p0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        p1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        with torch.cuda.stream(cap_stream):
            for k in range(steps):
                buf.copy_(packs[k % nsteps])
                p0[k].record(cap_stream)
                g2.replay()
                p1[k].record(cap_stream)
        torch.cuda.synchronize()
        phased = {"shift_ms_mean": statistics.mean(a.elapsed_time(z) for a, z in zip(p0, p1)),
                  "launches_per_shift": B.launches(), "form": "the same shift as separate launches, one graph"}
        B.set_single_launch(True)
    # accuracy on a sample of windows after the distinct shifts
    err = {}
    if rank == 0:
        import oracle
        B2 = None
        with torch.cuda.stream(cap_stream):
            B2 = CumWinBatch(ns, ds, Ts, b, p, args.precision, device=dev)
            B2.fill(firsts)
            for k in range(nsteps):
                B2.push(packs[k])
        torch.cuda.synchronize()
        for i in range(0, 512, 97):
            Xw = streams[i].rows(nsteps * p, nsteps * p + Ts[i])
            cen = oracle.center(Xw)
            e = {}
            for s_ in range(1, ds[i] + 1):
                tup = oracle.sample_sorted_tuples(ns[i], s_, 100, seed=i + s_)
                idx = np.array([oracle.storage_index(ns[i], b, t) for t in tup])
                ref = oracle.cumulant_tuples(Xw, tup, centred=cen)
                with torch.cuda.stream(cap_stream):
                    got = B2.cumulants(i, s_)
                torch.cuda.synchronize()
                got = got.cpu().numpy()[idx]
                e[str(s_)] = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
            err[f"window{i}(n={ns[i]},d={ds[i]})"] = e
        B2.close()
    mean_ms = ranks.max_over_ranks([statistics.mean(ms)], dev, world)[0]
    value = ranks.job_rate(world, 512, mean_ms * 1e-3)
    if rank == 0:
        from paper_1701_06446_gb300 import layout_size
        fifo = B.fifo
        elems = sum(layout_size(n_, b, s_) for n_, d_ in zip(ns, ds) for s_ in range(1, d_ + 1))
        # FP64 flops of the recovery per shift (as for one window: subset recursion, scaling, norm, fold)
        rec_flops = sum((2.0 * (2 ** (s_ - 1) - 1) + 5.0) * layout_size(n_, b, s_)
                        for n_, d_ in zip(ns, ds) for s_ in range(1, d_ + 1))
        # bytes per stored element: FP64 sum read + write (16), cumulant write (8), the FP32 workspace
        # write + read (8) and the FIFO slot read + write (8), or the leaving workspace's (8)
        bpe = 40
        peaks, peak_kind = _peaks()
        t_s = mean_ms * 1e-3
        whole = "one shift (the graph: staging, operand build, GEMM, fused recovery), timed as a whole"
        fp64_peak = fp64_peak_tflops(dev)
        roof = {"kernel": whole, "bound": "alu", "achieved": rec_flops / t_s / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": rec_flops / t_s / 1e12 / fp64_peak,
                "peak_kind": "measured FP64 (cuBLAS DGEMM 4096^3 in this run)", "traffic": None,
                "avg_launch_ms": mean_ms,
                "per_launch": f"{rec_flops:.4g} algorithmic FP64 flops of the recovery (per stored element of "
                              f"order s: 2(2^(s-1)-1) subset recursion + 1 scaling + 2 norm + 2 fold) over "
                              f"{elems} stored elements"}
        roof_hbm = {"kernel": whole, "bound": "hbm", "achieved": elems * bpe / t_s / 1e9,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": elems * bpe / t_s / 1e9 / peaks["hbm_gbs"], "peak_kind": f"{peak_kind} HBM copy",
                    "traffic": None, "avg_launch_ms": mean_ms,
                    "per_launch": f"{elems * bpe:.4g} algorithmic bytes ({bpe} per stored element: FP64 sum "
                                  f"read + write, cumulant write, FP32 workspace and "
                                  f"{'FIFO slot' if fifo else 'leaving workspace'} write + read)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": f"{args.precision}x3+f32acc+f64sum", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "windows": 512, "n": "U{8..64}", "orders": "1..{3,4}",
                       "b": b, "T": "U{2^12,2^14}", "p": p, "precision": args.precision,
                       "l2": "inputs and state larger than L2 (GB of sums), no flush",
                       "launch": "one CUDA graph per shift", "ksplit": ksplit, "tiles": B.tiles()},
            "batch": {"phase_by_phase": phased, "shift_ms_mean": mean_ms, "shift_ms_p50": lat[len(lat) // 2],
                      "shift_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "replays": reps,
                      "windows": 512, "state_elements": int(sum(
                          sum(__import__("paper_1701_06446_gb300").layout_size(n_, b, s_)
                              for s_ in range(1, d_ + 1)) for n_, d_ in zip(ns, ds)))},
            "error_vs_oracle": {"metric": "relative Frobenius error per order on 100 sampled tuples",
                                "windows": err},
            "roofline": roof, "roofline_other": roof_hbm,
            "gpu_launches": launches_per_shift * steps, "clocks": clocks,
            "setup_s": t_gen,
        }
        print(json.dumps(line), flush=True)
    B.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "bf16", "fp16"], default="bf16")
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="shifts of the FP64 GPU form measured for comparison (0: skip)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + [BATCH_WORKLOAD])
    ap.add_argument("--ref-tuples", type=int, default=1000,
                    help="seeded tuples of each order >= 3 timed per step of the reference arm")
    ap.add_argument("--cpu-tuples", type=int, default=5000,
                    help="seeded tuples of each order >= 4 in the cpu_baseline leg (orders <= 3 in full)")
    ap.add_argument("--grad", action="store_true", help="time forward + backward (adjoint) instead of shifts")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="override the workload's variable count")
    ap.add_argument("--window", type=int, default=None, help="override the workload's window length T")
    ap.add_argument("--shift", type=int, default=None, help="override the workload's shift size p")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = ranks.rank_env()
    if args.workload == BATCH_WORKLOAD:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm covers the "
                              "single-window workloads"}), flush=True)
            return
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
        ranks.init(world, "nccl")
        try:
            run_batch(args, rank, world)
        finally:
            ranks.finish(world)
        return
    W = WORKLOADS[args.workload]
    if args.n or args.window or args.shift:  # a smaller variant of the workload (profiling captures)
        import dataclasses
        n, T, p = args.n or W.n, args.window or W.T, args.shift or W.p
        W = dataclasses.replace(W, name=f"n{n}_d{W.d}_b{W.b}_T{T}_p{p}" + ("_ica" if W.kind == "ica_mix" else ""),
                                n=n, T=T, p=p, length=max(W.length, T + 64 * p))
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 only
        run_reference(args, W, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
    ranks.init(world, "nccl")
    try:
        (run_grad if args.grad else run_ours)(args, W, rank, world)
    finally:
        ranks.finish(world)


if __name__ == "__main__":
    main()
