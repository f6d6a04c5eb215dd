"""Replica sharding across GPUs: every rank analyses its own ladders.

CTUs, frames and ladders are independent (the motion-vector predictor is
(0,0) and a dependent rung reads only its own frame's reference decisions),
so N GPUs run N replicas with no collective on the data path.  The only
collectives are the barrier around the timed region and the max over ranks
of the measured time, from which the whole-job rate is computed (weak
scaling: each rank's work is fixed).  One process per GPU; the rendezvous
comes from the environment (torchrun: RANK, WORLD_SIZE, LOCAL_RANK,
MASTER_ADDR, MASTER_PORT).
"""
from __future__ import annotations

import os


def env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def seed_base(rank: int, base: int = 1000) -> int:
    """First seed of a rank's synthetic ladders: ranks never share content."""
    return base * (rank + 1)


def init(backend: str):
    """Joins the process group when there is more than one rank."""
    import torch.distributed as dist
    rank, world, _ = env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend, init_method="env://")
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The largest of every rank's value (e.g. its timed-region duration)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * world / seconds_max


def finish():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
