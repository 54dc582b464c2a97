"""Multi-GPU bookkeeping of the benchmark: one process per GPU, independent
work per rank (replicas of one solve, or disjoint shares of a problem set),
no collective on the data path.  The only communication is timing: a
barrier around the timed region and the slowest rank's time, so the
whole-job rate is (units of all ranks) / (max over ranks of the time).

Everything here takes a torch.distributed process group (NCCL on the GPU
box, gloo in the CPU tests) or none for a single process."""
from __future__ import annotations

import os


def env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous share of n_items for `rank`: sizes differ by at most one,
    every item belongs to exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def barrier(dist=None):
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_rate(local_units: float, local_seconds: float, dist=None, device=None):
    """Whole-job rate: units summed over ranks / the slowest rank's time.
    Returns (rate, max_seconds, total_units)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_units / local_seconds, local_seconds, local_units
    import torch

    t = torch.tensor([local_seconds, local_units], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t[1:].clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tsum.item()) / float(tmax.item()), float(tmax.item()), float(tsum.item())
