"""Independent replicas across ranks (one process per GPU, launched by torchrun).

The lattice Boltzmann path needs no data exchange between replicas, so the only
cross-rank operations are control: a barrier around the timed region, the
slowest rank's time, and the total of the units every rank processed. Ranks
read RANK, LOCAL_RANK and WORLD_SIZE from the environment.
"""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str):
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _reduce(value: float, op, device):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX if dist.is_available() else None, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM if dist.is_available() else None, device)


def seed_for_rank(base: int, rank: int) -> int:
    """Each rank's replica draws its own noise: seed base + rank."""
    return base + rank


def weak_scaling_value(local_units: float, local_seconds: float, device="cpu") -> float:
    """All ranks' units per second of the slowest rank (units / 1e6, e.g. MLUPS)."""
    total = sum_over_ranks(local_units, device)
    slowest = max_over_ranks(local_seconds, device)
    return total / slowest / 1e6
