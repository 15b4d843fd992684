"""Data-parallel replicas of the path across GPUs (one process per GPU).

Every configuration is independent, so N GPUs each evaluate their own batch
of the same size (weak scaling) and exchange nothing on the data path; the
only collective is the max of the per-rank step times, taken once after
timing.  Host-side logic only; ranks come from the usual torchrun
environment (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR/PORT).
"""
from __future__ import annotations

import os

from . import synth


def dist_env():
    """(world, rank, local_rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def rank_batch(workload, rank: int):
    """The rank's own configurations: rank 0 keeps the workload's batch,
    rank r > 0 draws a batch of the same size from seed 1000 + r."""
    if rank == 0:
        return workload.q
    return synth.make_q(1000 + rank, workload.n)


def max_over_ranks(value: float, pg=None, device=None) -> float:
    """Max of a per-rank scalar over the process group (identity alone)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, n_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job configurations per second: all ranks' work over the
    slowest rank's time."""
    return world * n_per_rank * steps / seconds
