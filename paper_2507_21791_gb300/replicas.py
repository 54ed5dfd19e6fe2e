"""Rank bookkeeping for runs on several GPUs of one node.

A run on N GPUs is one process per GPU: either N independent factorizations
(replicas: no collective on the data path) or one row-partitioned factorization
(rows.py: one all-gather per synchronization).  This module holds the host-side
pieces both share: the process's place in the run, the slowest rank's time (all
ranks report the max) and the whole-job throughput (units all ranks processed /
that time, weak scaling).
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device="cpu") -> float:
    """The maximum of x over the ranks of the initialized process group (x
    itself without one); device is where the backend reduces (cuda for NCCL)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world: int, bytes_per_rank: float, ms_max: float) -> float:
    """GB/s of the whole job: the bytes of all ranks over the slowest rank's time."""
    return world * bytes_per_rank / (ms_max * 1e-3) / 1e9
