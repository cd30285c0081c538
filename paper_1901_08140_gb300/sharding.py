"""Multi-GPU host logic: the path shards by particle id.

Electrons never interact (the paper neglects Coulomb forces between them),
and every random number is keyed by (swarm seed, particle id, step), so a
swarm split into id ranges over ranks gives the same electrons as one run.
Each rank runs its own range with no data-path collective; a step's time is
the maximum over ranks and its work the sum over ranks.
"""
from __future__ import annotations

from typing import Tuple


def id_range(rank: int, world: int, n_total: int) -> Tuple[int, int]:
    """[first, last) particle ids of `rank` when n_total electrons are split over `world` ranks."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(int(n_total), int(world))
    first = rank * base + min(rank, extra)
    return first, first + base + (1 if rank < extra else 0)


def weak_offset(rank: int, n_per_rank: int) -> int:
    """First id of `rank` when every rank runs n_per_rank electrons (weak scaling)."""
    return int(rank) * int(n_per_rank)


def reduce_step(ms: float, units: float, group=None) -> Tuple[float, float]:
    """(max step time over ranks, total units over ranks) with torch.distributed."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(ms), float(units)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
