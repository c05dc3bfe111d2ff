"""One stream on several GPUs: block shards of the top order over ranks.

Every rank holds a ``CumWin`` created as shard ``rank`` of ``world``
(``cumwin_create_shard``): the same samples enter every rank, each rank
updates and recovers the stored blocks of the top order d in its contiguous
range of lexicographic block ranks, and the orders below d are kept whole on
every rank.  The exchange steps are the ones the method has once the blocks
are split:

* a shift's p new rows are broadcast from one rank (``push(x, src)``);
* ``||C_d||^2`` is the sum of the ranks' partial sums over their blocks (an
  all-reduce of one double), after which the library forms ||C_s|| and nu_s
  (``cumwin_estimators_from_fro2``);
* reading C_d whole gathers the ranks' block ranges (an all-gather).

The per-rank object (``shard``) must offer ``fill(X)``, ``push(x)``,
``norms_device()`` (the d squared norms, order d as the rank's partial sum)
and ``cumulants(order)`` (block layout, order d valid in the rank's range);
by default it is the library's ``CumWin`` shard on the rank's GPU.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import CumWin, estimators_from_fro2, layout_size, shard_blocks


class ShardedCumWin:
    def __init__(self, n: int, d: int, b: int, T: int, p: int, precision: str = "bf16",
                 group=None, device=None, shard=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.n, self.d, self.b, self.T, self.p = n, d, b, T, p
        self.blocks = [shard_blocks(n, b, d, r, self.world) for r in range(self.world)]
        self.bs = b ** d
        self.h = shard if shard is not None else CumWin(n, d, b, T, p, precision, device=device,
                                                        shard=self.rank, nshards=self.world)

    def close(self):
        if hasattr(self.h, "close"):
            self.h.close()

    def fill(self, X: torch.Tensor, src: int = 0):
        """The first window, valid on rank `src`; broadcast to every rank."""
        X = X.contiguous()
        dist.broadcast(X, src=src, group=self.group)
        self.h.fill(X)

    def push(self, x: torch.Tensor, src: int = 0):
        """One shift: the p new rows (valid on rank `src`) are broadcast, then every
        rank updates its own blocks."""
        x = x.contiguous()
        dist.broadcast(x, src=src, group=self.group)
        self.h.push(x)

    def norms(self) -> tuple[np.ndarray, np.ndarray]:
        """(||C_s||, nu_s), s = 1..d, of the whole window on every rank."""
        fro2 = self.h.norms_device().clone()
        top = fro2[self.d - 1:self.d].contiguous()
        dist.all_reduce(top, op=dist.ReduceOp.SUM, group=self.group)
        fro2[self.d - 1:self.d] = top
        return estimators_from_fro2(fro2.cpu().numpy())

    def cumulants(self, order: int) -> torch.Tensor:
        """C_order in the block layout on every rank (order d gathered from the ranks' ranges)."""
        C = self.h.cumulants(order)
        if order < self.d:
            return C
        lo, hi = self.blocks[self.rank]
        width = max(e - s for s, e in self.blocks) * self.bs
        part = torch.zeros(width, dtype=C.dtype, device=C.device)
        part[: (hi - lo) * self.bs] = C[lo * self.bs: hi * self.bs]
        parts = [torch.empty_like(part) for _ in range(self.world)]
        dist.all_gather(parts, part, group=self.group)
        out = torch.empty(layout_size(self.n, self.b, order), dtype=C.dtype, device=C.device)
        for (s, e), q in zip(self.blocks, parts):
            out[s * self.bs: e * self.bs] = q[: (e - s) * self.bs]
        return out
