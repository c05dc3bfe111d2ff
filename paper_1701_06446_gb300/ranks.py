"""Rank plumbing of the multi-GPU benchmark (weak scaling).

The workloads are independent streams, so the path shards without a data-path
collective: one process per GPU, each advancing its own disjoint stretch of
the stream.  The only communication is a barrier on each side of the timed
region and the maximum over ranks of the elapsed times; the whole-job rate is
the units all ranks processed divided by that maximum.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init(world: int, backend: str) -> None:
    """Join the process group (rendezvous from MASTER_ADDR / MASTER_PORT) when world > 1."""
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)


def finish(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def stream_base(rank: int, T: int, p: int, shifts: int) -> int:
    """First stream row of a rank's stretch: a window of T rows, `shifts` shifts of p
    rows, and one shift of gap, so that the ranks' stretches are disjoint."""
    return rank * (T + (shifts + 1) * p)


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(values, device, world: int) -> list[float]:
    """Element-wise maximum over ranks of a list of floats (float64 on `device`)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job rate: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds_max
