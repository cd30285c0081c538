"""Multi-GPU host logic: the path shards by particle id.

Electrons never interact (the paper neglects Coulomb forces between them),
and every random number is keyed by (swarm seed, particle id, step), so a
swarm split into id ranges over ranks gives the same electrons as one run.
Each rank runs its own range with no data-path collective; a step's time is
the maximum over ranks and its work the sum over ranks.  The one exchange,
when a swarm is split over ranks, is the FP64 sum of its tally group sums
(two all-reduces: pass 1, then pass 2 about the drift the merged pass 1
gives), after which every rank holds the tallies of the whole swarm.
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


def _all_reduce_sum(a, group=None):
    """FP64 sum over ranks of a host array (the collective of the merge)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return np.asarray(a, dtype=np.float64)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def merge_tallies(sums1, sums2_about, e_over_n_Td, n_total_m3, nu_trial=0.0, n_spawned=0, n_capped=0,
                  error_flags=0, group=None):
    """Tallies of one swarm whose electrons ran on several ranks.

    sums1: this rank's pass-1 group sums (32 x 21); sums2_about(drift): this
    rank's pass-2 group sums (32 x 8) about a drift vector.  Every rank calls
    this; all get the same result.
    """
    from . import bz
    g1 = _all_reduce_sum(sums1, group)
    drift = bz.drift_from_group_sums(g1)
    g2 = _all_reduce_sum(sums2_about(drift), group)
    counts = _all_reduce_sum([float(n_spawned), float(n_capped)], group)
    flags = int(error_flags)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
            bits = _all_reduce_sum([float((flags >> b) & 1) for b in range(8)], group)
            flags = sum(1 << b for b in range(8) if bits[b] > 0)
    except ImportError:
        pass
    return bz.finalize_group_sums(g1, g2, e_over_n_Td, n_total_m3, nu_trial, int(counts[0]), int(counts[1]), flags)
