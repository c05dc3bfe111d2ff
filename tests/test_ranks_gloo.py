"""The multi-rank path of the benchmark on CPU: two `gloo` ranks, each advancing
its own stretch of the stream (weak scaling, no data-path collective), with the
barrier and the maximum over ranks that the timing uses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1701_06446_gb300 import ranks
from paper_1701_06446_gb300.streams import WORKLOADS


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    r, w, lr = ranks.rank_env()
    assert (r, w, lr) == (rank, world, rank)
    ranks.init(w, "gloo")
    try:
        W = WORKLOADS["n4_d4_b2_T1000_p100"]
        shifts = 7
        base = ranks.stream_base(r, W.T, W.p, shifts)
        spans = [None] * w
        dist.all_gather_object(spans, (base, base + W.T + shifts * W.p))
        spans.sort()
        for (a0, a1), (b0, _) in zip(spans, spans[1:]):
            assert a1 <= b0, spans  # disjoint stretches
        # each rank's window after its shifts, and its order-2 cumulants from the oracle
        X = W.stream().rows(base + shifts * W.p, base + shifts * W.p + W.T)
        c2 = oracle.cumulants(X, 2, W.b)[1]
        got = [None] * w
        dist.all_gather_object(got, c2.tolist())
        assert not np.allclose(got[0], got[1])  # independent streams
        assert np.array_equal(np.array(got[r]), c2)
        ranks.barrier(w)
        # the timing reductions: maximum over ranks, whole-job rate
        m = ranks.max_over_ranks([1.5 + r, 10.0 - r], torch.device("cpu"), w)
        assert m == [1.5 + (w - 1), 10.0]
        assert ranks.job_rate(w, 50, m[0]) == pytest.approx(w * 50 / m[0])
    finally:
        ranks.finish(w)


def test_two_gloo_ranks_weak_scaling_plumbing():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_single_rank_needs_no_process_group():
    os.environ.pop("WORLD_SIZE", None)
    r, w, _ = ranks.rank_env()
    ranks.init(w, "gloo")  # no-op
    assert ranks.max_over_ranks([3.0], torch.device("cpu"), w) == [3.0]
    ranks.barrier(w)
    ranks.finish(w)
    assert ranks.stream_base(0, 100, 10, 5) == 0
    assert ranks.stream_base(1, 100, 10, 5) == 160
