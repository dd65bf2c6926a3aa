"""Environment replicas over ranks: the multi-GPU form of the batched step.

Environments never interact (Sec. 3.2 advances the agents of each scene
instance on its own), so N GPUs run N independent batches: rank r builds the
batch with seed r, steps it with no collective on the data path, and only
the timing meets at the end (the largest time over the ranks, the sum of
agent-steps).  One process per GPU, torch.distributed for that last exchange
(NCCL on GPUs, gloo on the host).
"""
from __future__ import annotations

import os


def dist_env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(rank: int) -> int:
    """Seed of rank r's batch: distinct per rank, rank 0 = the 1-GPU batch."""
    return int(rank)


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "sum", device)


def aggregate_throughput(agent_steps: float, seconds: float, device=None) -> float:
    """Whole-job agent-steps/s: every rank's agent-steps over the slowest
    rank's time (weak scaling: per-rank work is fixed as ranks are added)."""
    total = sum_over_ranks(agent_steps, device)
    slowest = max_over_ranks(seconds, device)
    return total / slowest
