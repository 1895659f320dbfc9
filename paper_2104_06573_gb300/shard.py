"""Event sharding across ranks: one process per GPU, no data-path collective.

Events are independent units of work (each event's hits are reconstructed on their own, §3), so
N GPUs split the event stream and never exchange data on the hot path.  The only cross-rank
operations are host-side: a barrier around a timed region, the maximum of the ranks' durations
(the job's time is the slowest rank's), and an optional gather of results onto rank 0.

Two ways to split:
  * `shard(n, rank, world)`: a fixed event list dealt round-robin (strong scaling of one list);
  * `rank_seed0(rank)`: each rank draws its own batch from a disjoint seed range (weak scaling,
    per-GPU work fixed as N grows), which is what the benchmark times.
"""
from __future__ import annotations

import numpy as np

SEED_STRIDE = 100000


def shard(n_events: int, rank: int, world: int) -> np.ndarray:
    """Indices of the events rank `rank` of `world` processes (round-robin, disjoint, covering)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    return np.arange(rank, n_events, world, dtype=np.int64)


def rank_seed0(rank: int) -> int:
    """First event seed of rank `rank`'s own batch; ranks' seed ranges do not overlap."""
    return rank * SEED_STRIDE


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def barrier() -> None:
    d = _dist()
    if d is not None and d.get_world_size() > 1:
        d.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (identity without a process group).  `device` is the
    rank's CUDA device under NCCL and None (CPU tensor) under gloo."""
    d = _dist()
    if d is None or d.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj):
    """Every rank's `obj` as a list on rank 0 (rank order), None on the other ranks."""
    d = _dist()
    if d is None or d.get_world_size() == 1:
        return [obj]
    out = [None] * d.get_world_size() if d.get_rank() == 0 else None
    d.gather_object(obj, out, dst=0)
    return out
