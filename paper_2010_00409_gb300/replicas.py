"""Replica bookkeeping for runs on several GPUs.

The focal-field job does not shard (every configuration fits one GB300), so N
GPUs run N independent replicas with no data-path collective.  Ranks only agree
on which independent units each one owns and on the slowest rank's time; the
whole-job rate is the work of all ranks over that time.
"""
from __future__ import annotations


def env():
    """(world_size, rank, local_rank) from the torch.distributed launcher's env."""
    import os
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def units_for_rank(n_units: int, world: int, rank: int) -> list[int]:
    """Independent unit ids (e.g. pulse realisations) owned by `rank`: a
    round-robin split, so every unit has exactly one owner."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    return list(range(rank, n_units, world))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(work_per_rank: float, world: int, t_max_s: float) -> float:
    """Aggregate throughput: all ranks' work over the slowest rank's time."""
    if t_max_s <= 0:
        raise ValueError("time must be positive")
    return work_per_rank * world / t_max_s
