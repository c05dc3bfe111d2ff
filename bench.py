"""Benchmark: window updates/s of the sliding-window cumulant path on GB300.

One step = one window shift of the whole hot path: ring append / X_(-)
extraction, moment-sum update of orders 1..d, moment-to-cumulant recovery of
orders 1..d, and the norm reduction (Algorithm 1, one loop iteration).

Default workload: n=60 variables, orders 1..4, block size 3, window T=2^15,
shift p=2^10, FP32 samples (Gaussian, then a Gaussian copula with
exponential(1) marginals), seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|bf16]
    python bench.py --impl reference      # the CPU oracle on the same workload

Prints one JSON line (rank 0).  Under torchrun each rank advances its own
independent stream (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
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
DEFAULT_WORKLOAD = "n60_d4_b3_T32768_p1024"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (CUDA cores), nominal


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def algorithmic_flops(W, fifo: bool = False) -> dict:
    """Flops of one shift: update 2 * K * E_s per order (one product per
    multiply-add) with K = 2p samples (entering and leaving), or K = p when
    the leaving batch's sums come from the batch-sum FIFO; recovery
    2 * (2^{s-1} - 1) * E_s (one multiply-add per subset term)."""
    from paper_1701_06446_gb300 import layout_size
    K = W.p if fifo else 2 * W.p
    upd = sum(2.0 * K * layout_size(W.n, W.b, s) for s in range(1, W.d + 1))
    rec = sum(2.0 * (2 ** (s - 1) - 1) * layout_size(W.n, W.b, s) for s in range(2, W.d + 1))
    # the recovery launch(es) as a whole, FP64: per stored element of order s the subset
    # recursion (2 per term), the 1/T scaling (1), multiplicity * C^2 (2) and the fold of the
    # shift's batch sums into S_s (2)
    rec_launch = sum((2.0 * (2 ** (s - 1) - 1) + 5.0) * layout_size(W.n, W.b, s) for s in range(1, W.d + 1))
    return {"update": upd, "recovery": rec, "recovery_launch": rec_launch}


# DRAM bytes (read + write) per launch of the recovery from one ncu capture of the current
# kernel (see profiles/), by workload; None where no capture of the current kernel exists.
RECOVERY_TRAFFIC = {"n60_d4_b3_T32768_p1024": 13002496}
# the same for the GEMM (k_kr_gemm)
GEMM_TRAFFIC = {"n60_d4_b3_T32768_p1024": 15818240}


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

def oracle_sample_time(X: np.ndarray, W, per_order: int, seed: int) -> tuple[float, str]:
    """Seconds one full oracle recomputation of C_1..C_d for window X would take,
    from timing every sorted tuple of orders <= 2 and `per_order` seeded
    sorted tuples of each higher order (extrapolated linearly by tuple count)."""
    import oracle
    t0 = time.perf_counter()
    cen = oracle.center(X)
    total = time.perf_counter() - t0
    parts = []
    for s in range(1, W.d + 1):
        n_tuples = math.comb(W.n + s - 1, s)
        if s <= 2 or n_tuples <= per_order:
            import itertools
            tup = np.array(list(itertools.combinations_with_replacement(range(W.n), s)), np.int32)
            t0 = time.perf_counter()
            oracle.cumulant_tuples(X, tup, centred=cen)
            total += time.perf_counter() - t0
            parts.append(f"order {s}: all {n_tuples}")
        else:
            tup = oracle.sample_sorted_tuples(W.n, s, per_order, seed + s)
            t0 = time.perf_counter()
            oracle.cumulant_tuples(X, tup, centred=cen)
            dt = time.perf_counter() - t0
            total += dt * n_tuples / per_order
            parts.append(f"order {s}: {per_order} of {n_tuples} tuples, extrapolated")
    return total, "; ".join(parts)


def oracle_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, W, rank: int):
    if rank != 0:
        return
    X = W.stream().rows(0, W.T).astype(np.float64)
    for _ in range(args.warmup):
        oracle_sample_time(X, W, 100, seed=0)
    secs = []
    sample = ""
    for k in range(args.steps):
        dt, sample = oracle_sample_time(X, W, args.ref_tuples, seed=k)
        secs.append(dt)
    per = statistics.mean(secs)
    value = 1.0 / per
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(W, "fp64-oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": f"full recomputation of one window from scratch per step; {sample}"},
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
    """The plain FP64 GPU form on the same stretch of the stream, for comparison."""
    import torch
    from paper_1701_06446_gb300 import CumWin
    X = torch.from_numpy(stream.rows(base, base + W.T + (steps + 3) * W.p)).to(dev)
    h = CumWin(W.n, W.d, W.b, W.T, W.p, "fp64", device=dev)
    h.fill(X[: W.T])
    for k in range(3):
        h.push(X[W.T + k * W.p: W.T + (k + 1) * W.p])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.set_timing(True)
    e0.record()
    for k in range(3, 3 + steps):
        h.push(X[W.T + k * W.p: W.T + (k + 1) * W.p])
    e1.record()
    torch.cuda.synchronize()
    t = h.get_timing()
    h.close()
    ms = e0.elapsed_time(e1) / steps
    upd = t["update_ms"] / max(t["shifts"], 1)
    return {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "update_ms": upd,
            "update_tflops": algorithmic_flops(W)["update"] / (upd * 1e-3) / 1e12, "steps": steps}


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

    # end-to-end through the C ABI with host buffers: H2D of X_(+) from pinned memory and D2H of
    # every step's squared norms and status inside the timed region.  Streaming form: each push's
    # norms are enqueued behind its recovery (which overlaps the next push) and nu is formed on the
    # host once the loop has been synchronised.  Synchronous form: norms() blocks after every push.
    e2e_steps_total = (e2e_reps + 1) * e2e_steps
    host = torch.from_numpy(stream.rows(base + W.T + nsteps * W.p,
                                        base + W.T + (nsteps + e2e_steps_total) * W.p)).pin_memory()
    hb = [host[k * W.p:(k + 1) * W.p] for k in range(e2e_steps_total)]
    fro2_host = torch.zeros(e2e_steps, W.d, dtype=torch.float64).pin_memory()
    st_host = torch.full((e2e_steps,), -1, dtype=torch.int32).pin_memory()
    stream_s = []
    for r in range(e2e_reps):
        st_host.fill_(-1)
        torch.cuda.synchronize()
        ranks.barrier(world)
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            h.push_host(hb[r * e2e_steps + k])
            h.norms_enqueue(fro2_host[k], st_host[k:k + 1])
        h.join()
        torch.cuda.synchronize()
        fro_all = np.sqrt(fro2_host.numpy())
        nu_all = fro_all[:, 2:] / fro_all[:, 1:2] ** (0.5 * np.arange(3, W.d + 1)) if W.d >= 3 else None
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
    flops = algorithmic_flops(W, fifo)
    peaks, peak_kind = _peaks()
    rec_ms = timing["cumulant_ms"] / max(timing["shifts"], 1)  # timed region
    upd_ms = timing_split["update_ms"] / max(timing_split["shifts"], 1)  # instrumented pass
    stg_ms = timing_split["stage_ms"] / max(timing_split["shifts"], 1)
    if precision == "fp64":
        achieved = flops["update"] / (upd_ms * 1e-3) / 1e12
        roof = {"kernel": "k_update_f64", "bound": "alu", "achieved": achieved,
                "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS,
                "peak_kind": "nominal FP64 (CUDA cores)", "traffic": None,
                "per_launch": f"{flops['update']:.4g} algorithmic flops (2 x 2p x E_s summed over orders)",
                "avg_launch_ms": upd_ms}
        roof_other = None
    else:
        achieved = flops["update"] / (upd_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        roof_gemm = {"kernel": "k_kr_gemm", "bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} bf16 sustained (of measured)",
                     "traffic": GEMM_TRAFFIC.get(W.name), "avg_launch_ms": upd_ms,
                     "share_of_step": upd_ms / ms_per_step,
                     "per_launch": f"{flops['update']:.4g} algorithmic flops (2 x K x E_s summed over "
                                   f"orders, K = {'p: entering samples; leaving sums from the FIFO' if fifo else '2p'}); "
                                   f"the tensor pipe issues 3x (hi*hi + hi*lo + lo*hi)"}
        rec_achieved = flops["recovery_launch"] / (rec_ms * 1e-3) / 1e12
        roof_rec = {"kernel": "k_recover_fused" if W.d <= 4 else
                    "recovery (k_recover_fused, k_split, k_cumulants<5..d>, k_norm_final)",
                    "bound": "alu", "achieved": rec_achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": rec_achieved / FP64_NOMINAL_TFLOPS,
                    "peak_kind": "nominal FP64 rate (the recovery's scarcest pipe)",
                    "traffic": RECOVERY_TRAFFIC.get(W.name), "avg_launch_ms": rec_ms,
                    "share_of_step": rec_ms / ms_per_step,
                    "per_launch": f"{flops['recovery_launch']:.4g} algorithmic FP64 flops (per stored element "
                                  f"of order s: 2(2^(s-1)-1) subset recursion + 1 scaling + 2 norm + 2 fold)"}
        if W.d >= 5:
            roof_rec["note"] = ("orders >= 5 form their subset products in two-word FP32 arithmetic on the "
                                "FMA pipe, so these FP64-class flops can run faster than the FP64 pipe's peak")
        # the roofline line is the dominant kernel's; the other is kept beside it
        if rec_ms >= upd_ms:
            roof, roof_other = roof_rec, roof_gemm
        else:
            roof, roof_other = roof_gemm, roof_rec
    cpu = None
    fp64_form = None
    if precision != "fp64" and args.fp64_steps > 0:
        fp64_form = measure_fp64_form(W, stream, base, args.fp64_steps, dev)
    if world == 1 and not args.no_cpu_baseline:
        Xw = final.astype(np.float64)
        secs, sample = oracle_sample_time(Xw, W, args.ref_tuples, seed=7)
        cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": f"full recomputation of one window; {sample}"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == "fp64" else f"{precision}x3+f32acc+f64sum",
        "data": "synthetic", "config": dict(config_of(W, precision), ksplit=ksplit, fifo=fifo),
        "samples_per_s": value * W.p,
        "tflops": flops["update"] / (ms_per_step * 1e-3) / 1e12,
        "stage_ms": stg_ms, "update_ms": upd_ms, "recovery_ms": rec_ms,
        "fp64_form": fp64_form,
        "error_vs_oracle": {"metric": "relative Frobenius error per order on 200 sampled tuples",
                            "per_order": err},
        "roofline": roof, "roofline_other": roof_other, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": W.p * W.n * 4,
                "d2h_bytes_per_step": W.d * 8 + 4, "steps": e2e_steps, "loops": e2e_reps,
                "form": "push_host + norms_enqueue per step (recovery pipelined with the next push), "
                        "one synchronisation at the end of each loop; no L2 flush; median of the loops",
                "synchronous": {"value": e2e_sync_value, "unit": UNIT,
                                "form": "push_host + blocking norms() per step"}},
        "gpu_launches": timing["launches"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    h.close()


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
        roof = {"kernel": whole, "bound": "alu", "achieved": rec_flops / t_s / 1e12, "peak": FP64_NOMINAL_TFLOPS,
                "unit": "TFLOP/s", "frac": rec_flops / t_s / 1e12 / FP64_NOMINAL_TFLOPS,
                "peak_kind": "nominal FP64 rate (the recovery's scarcest pipe)", "traffic": None,
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
                       "launch": "one CUDA graph per shift", "ksplit": ksplit},
            "batch": {"shift_ms_mean": mean_ms, "shift_ms_p50": lat[len(lat) // 2],
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
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="shifts of the FP64 GPU form measured for comparison (0: skip)")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + [BATCH_WORKLOAD])
    ap.add_argument("--ref-tuples", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 only
        run_reference(args, W, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
    ranks.init(world, "nccl")
    try:
        run_ours(args, W, rank, world)
    finally:
        ranks.finish(world)


if __name__ == "__main__":
    main()
