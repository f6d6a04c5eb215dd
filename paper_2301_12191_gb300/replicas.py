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
import socket
import subprocess
import sys


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


def sum_over_ranks(value: float, device=None) -> float:
    """The sum of every rank's value (e.g. the units it processed)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * world / seconds_max


def finish():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch_command(script: str, argv, n: int, port: int | None = None):
    """Command line that runs `script argv` as n ranks of one node: one
    process per GPU, rendezvous on 127.0.0.1 (each rank reads RANK,
    LOCAL_RANK and WORLD_SIZE from its environment)."""
    port = port or free_port()
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={int(n)}",
            "--master-addr", "127.0.0.1", f"--master-port={port}", script, *argv]


def spawn(script: str, argv, n: int, **kw) -> subprocess.CompletedProcess:
    """Runs `script argv` as n ranks (launch_command) and waits for them."""
    return subprocess.run(launch_command(script, argv, n), **kw)
