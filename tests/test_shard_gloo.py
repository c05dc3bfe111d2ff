"""Block shards of one stream over two ranks, on CPU with `gloo`.

``ShardedCumWin`` broadcasts the samples from rank 0, sums the ranks' partial
squared norms of the top order (all-reduce) and gathers the top order's block
ranges (all-gather).  Here each rank's compute is a stand-in that evaluates
the oracle on the rank's shard (the block range the library assigns with
``cumwin_shard_blocks``): the orders below d whole, the top order on the
rank's blocks only, and the norm of the top order over those blocks.  The
gathered cumulants and the combined norms and nu must equal the oracle's on
the whole window: the partition covers every block exactly once and the
collectives put the pieces together.  (The library's own shards are checked
on one GPU in test_gpu_shards.py.)
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1701_06446_gb300 import layout_size, shard_blocks
from paper_1701_06446_gb300.streams import WORKLOADS


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleShard:
    """CPU stand-in for the library's shard `rank` of `world` (test only)."""

    def __init__(self, n, d, b, T, rank, world):
        self.n, self.d, self.b, self.T = n, d, b, T
        self.lo, self.hi = shard_blocks(n, b, d, rank, world)
        self.X = None

    def fill(self, X):
        self.X = X.numpy().astype(np.float64)

    def push(self, x):
        self.X = np.vstack([self.X[len(x):], x.numpy().astype(np.float64)])

    def _top(self):
        n, d, b = self.n, self.d, self.b
        bs = b ** d
        idx = oracle.block_elements(n, b, d)[self.lo * bs: self.hi * bs]
        out = np.zeros(layout_size(n, b, d))
        keep = np.all(idx < n, axis=1)
        if keep.any():
            vals = oracle.cumulant_tuples(self.X, np.sort(idx[keep], axis=1).astype(np.int32))
            part = np.zeros(idx.shape[0])
            part[keep] = vals
            out[self.lo * bs: self.hi * bs] = part
        return out

    def cumulants(self, order):
        if order < self.d:
            return torch.from_numpy(oracle.cumulants(self.X, self.d - 1, self.b)[order - 1])
        return torch.from_numpy(self._top())

    def norms_device(self):
        n, d, b = self.n, self.d, self.b
        fro2 = np.zeros(d)
        low = oracle.cumulants(self.X, d - 1, b) if d > 1 else []
        for s in range(1, d + 1):
            C = low[s - 1] if s < d else self._top()
            blocks = oracle.sorted_block_tuples(n, b, s)
            mult = np.repeat([oracle.block_multiplicity(j) for j in blocks], b ** s)
            fro2[s - 1] = float(np.sum(mult * C * C))
        return torch.from_numpy(fro2)


def _worker(rank, world, port, n, d, b, T, p, shifts, seed):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1701_06446_gb300.sharded import ShardedCumWin
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((n, n)) / np.sqrt(n)
        stream = (rng.standard_t(5, size=(T + shifts * p, n)) @ A + 0.3).astype(np.float32)
        sh = ShardedCumWin(n, d, b, T, p, group=None, shard=OracleShard(n, d, b, T, rank, world))
        # only rank 0 holds the samples; the others receive them by broadcast
        X = torch.from_numpy(stream[:T]) if rank == 0 else torch.zeros(T, n)
        sh.fill(X)
        for w in range(shifts):
            x = torch.from_numpy(stream[T + w * p: T + (w + 1) * p]) if rank == 0 else torch.zeros(p, n)
            sh.push(x)
        window = stream[shifts * p:]
        ref = oracle.cumulants(window, d, b)
        for s in range(1, d + 1):
            got = sh.cumulants(s).numpy()
            assert np.allclose(got, ref[s - 1], rtol=1e-12, atol=1e-14 * np.abs(ref[s - 1]).max()), (rank, s)
        fro, nu = sh.norms()
        ofro, onu = oracle.norms(window, d)
        assert np.allclose(fro, ofro, rtol=1e-12), (rank, fro, ofro)
        assert np.allclose(nu[2:], onu[2:], rtol=1e-12), (rank, nu, onu)
        # the ranks' ranges partition the top order's blocks
        ranges = [None] * world
        dist.all_gather_object(ranges, (sh.h.lo, sh.h.hi))
        assert ranges[0][0] == 0 and ranges[-1][1] == len(oracle.sorted_block_tuples(n, b, d))
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0 and a0 < a1 and b0 < b1
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("cfg", ["n4_d4", "ragged_d5"])
def test_two_gloo_ranks_block_shards_match_oracle(cfg):
    if cfg == "n4_d4":
        W = WORKLOADS["n4_d4_b2_T1000_p100"]
        args = (W.n, W.d, W.b, W.T, W.p, 3, 1)
    else:  # b does not divide n (padded variables), an odd number of top-order blocks
        args = (7, 5, 3, 200, 40, 3, 2)
    mp.spawn(_worker, args=(2, _free_port()) + args, nprocs=2, join=True)
