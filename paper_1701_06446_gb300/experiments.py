"""The paper's experiments, run through the library on the GPU.

* ``detection`` (Section 4.3): the stream of Section 4.2 at the paper's scale —
  n = 100 variables, window t = 10^6, shifts of t_up = 2.5e4, w = 1..61 — with
  ||C_2||, nu_3 and nu_4 of every window (Eqs. me, mef), and the 5th, 50th and
  95th percentiles of nu_4 over many streams at w = 1 (Gaussian window) and at
  w >= t/t_up + 1 = 41 (no Gaussian sample left).  The paper reports
  (0.004, 0.006, 0.011) and (0.199, 0.209, 0.220) over 100 streams.
* ``speedup`` (Section 3.3): the time of one sliding update of C_1..C_d
  against a full recalculation of the same window (`cumwin_recompute`), at the
  paper's window sizes and orders (t = 5e5 and 1e6 with d = 4, b = 4; 5e6 with
  d = 5, b = 3; 2.5e7 with d = 6, b = 2), next to the operation-count ratio
  t / (2 t_up + B(d)) of the complexity analysis (Eq. complxn).

Run as ``python -m paper_1701_06446_gb300.experiments detection`` or
``... speedup``; each prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import CumWin
from .streams import GaussThenTCopulaGPU


def bell(d: int) -> int:
    """Bell number B(d) (set partitions of d elements)."""
    row = [1]
    for _ in range(d):
        nxt = [row[-1]]
        for v in row:
            nxt.append(nxt[-1] + v)
        row = nxt
    return row[0]


def detection(seeds: int = 100, n: int = 100, T: int = 10 ** 6, p: int = 25000, wmax: int = 61, b: int = 4,
              precision: str = "bf16", nu: int = 10, device: str = "cuda") -> dict:
    import torch
    sat = T // p + 1  # first window without Gaussian samples
    curves = {"c2": [], "nu3": [], "nu4": []}
    nu4_w1, nu4_sat_first, nu4_sat_all = [], [], []
    t0 = time.perf_counter()
    with CumWin(n, 4, b, T, p, precision, device=device) as h:
        for sd in range(seeds):
            gen = GaussThenTCopulaGPU(n, first=T, seed=1000 + sd, nu=nu, device=device)
            h.fill(gen.take(T))
            c2, n3, n4 = [], [], []
            for w in range(1, wmax + 1):
                if w > 1:
                    h.push(gen.take(p))
                fro, nuv = h.norms()
                c2.append(float(fro[1]))
                n3.append(float(nuv[2]))
                n4.append(float(nuv[3]))
            torch.cuda.synchronize()
            if sd == 0:
                curves = {"c2": c2, "nu3": n3, "nu4": n4}
            nu4_w1.append(n4[0])
            if wmax >= sat:
                nu4_sat_first.append(n4[sat - 1])
                nu4_sat_all.extend(n4[sat - 1:])
    q = lambda v: [float(x) for x in np.percentile(v, [5, 50, 95])] if v else None
    return {
        "experiment": "detection", "n": n, "d": 4, "b": b, "T": T, "p": p, "wmax": wmax, "nu": nu,
        "precision": precision, "seeds": seeds, "seconds": time.perf_counter() - t0,
        "curves_seed0": curves,
        "nu4_quantiles_5_50_95": {"w=1": q(nu4_w1), f"w={sat}": q(nu4_sat_first), f"w>={sat}": q(nu4_sat_all)},
        "paper_quantiles_5_50_95": {"w=1": [0.004, 0.006, 0.011], f"w>={sat}": [0.199, 0.209, 0.220]},
    }


PAPER_SPEEDUP_CONFIGS = ((500000, 4, 4), (1000000, 4, 4), (5000000, 5, 3), (25000000, 6, 2))


def speedup(n: int = 24, configs=PAPER_SPEEDUP_CONFIGS, fractions=(100, 50, 20), reps: int = 5,
            precision: str = "bf16", device: str = "cuda") -> dict:
    import torch
    rows = []
    for (T, d, b) in configs:
        for frac in fractions:
            p = T // frac
            gen = torch.Generator(device=device)
            gen.manual_seed(T + d)
            X = torch.randn(T + (reps + 1) * p, n, generator=gen, device=device)
            with CumWin(n, d, b, T, p, precision, device=device) as h:
                h.fill(X[:T])
                h.push(X[T:T + p])  # warm-up
                torch.cuda.synchronize()
                st = torch.cuda.current_stream()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(st)
                for k in range(1, reps + 1):
                    h.push(X[T + k * p: T + (k + 1) * p])
                e1.record(st)
                h.recompute()
                e2.record(st)
                torch.cuda.synchronize()
                push_ms = e0.elapsed_time(e1) / reps
                rec_ms = e1.elapsed_time(e2)
            del X
            rows.append({"T": T, "d": d, "b": b, "n": n, "p": p, "push_ms": push_ms, "recompute_ms": rec_ms,
                         "speedup": rec_ms / push_ms, "model_t_over_2tup_plus_Bd": T / (2 * p + bell(d))})
    return {"experiment": "speedup", "precision": precision, "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("detection")
    a.add_argument("--seeds", type=int, default=100)
    a.add_argument("--n", type=int, default=100)
    a.add_argument("--T", type=int, default=10 ** 6)
    a.add_argument("--p", type=int, default=25000)
    a.add_argument("--wmax", type=int, default=61)
    a.add_argument("--precision", default="bf16")
    s = sub.add_parser("speedup")
    s.add_argument("--n", type=int, default=24)
    s.add_argument("--reps", type=int, default=5)
    s.add_argument("--precision", default="bf16")
    args = ap.parse_args(argv)
    if args.cmd == "detection":
        out = detection(args.seeds, args.n, args.T, args.p, args.wmax, precision=args.precision)
    else:
        out = speedup(args.n, reps=args.reps, precision=args.precision)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
