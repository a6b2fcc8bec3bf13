"""Multi-process layout of the simulation (one process per GPU).

RIRs are independent (Section 3: each is a sum over its own image sources),
so the work shards with no exchange step: a process either runs a replica of
a workload (weak scaling, what the benchmark measures) or takes a contiguous
range of the RIRs of a batch, and the host reassembles the ranges.  The only
collectives are on the host side of the measurement: the slowest rank's step
time and the reassembly of sharded outputs.  Everything here works with any
torch.distributed backend (gloo on CPU in the tests, NCCL on GPUs).
"""
from __future__ import annotations

from typing import List, Tuple


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) share of n items for `rank` of `world`: the first
    n % world ranks take one item more; shares are ordered by rank."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the slowest rank's step time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units per second of the whole job: all ranks' units over the slowest
    rank's time (replicas: every rank processes units_per_rank)."""
    if seconds_max <= 0:
        raise ValueError("time must be positive")
    return units_per_rank * world / seconds_max


def gather_shards(local, n_total: int, device=None):
    """Reassembles per-rank contiguous shards (first dimension, as given by
    shard_range) into the full [n_total, ...] tensor on every rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    world = dist.get_world_size()
    sizes = [shard_range(n_total, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=device)
    pad[:local.shape[0]] = local
    parts: List = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([parts[r][:hi - lo] for r, (lo, hi) in enumerate(sizes)], dim=0)
