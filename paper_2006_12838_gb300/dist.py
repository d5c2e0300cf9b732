"""Multi-process helpers for running the hot path on several GPUs of a node.

The PLIC batches and the VOF fields are independent units: a multi-GPU run
gives each rank its own units (weak scaling: contiguous cell ranges, or whole
fields balanced by their interface-cell counts) and needs no data-path
collective.  The only collectives are around the timing: a barrier before and
after the timed region and the maximum of the per-rank times.  Launch with
torchrun (one process per GPU); the env variables RANK / WORLD_SIZE /
LOCAL_RANK / MASTER_ADDR / MASTER_PORT select the process group.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None) -> bool:
    """Initialise the default process group when WORLD_SIZE > 1."""
    _, world, _ = rank_info()
    if world <= 1 or dist.is_initialized():
        return dist.is_initialized()
    dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))
    return True


def shard(n_units: int, rank: int, world: int):
    """Contiguous [start, stop) range of rank's share of n_units (sizes differ
    by at most one)."""
    base, rem = divmod(n_units, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)


def assign_fields(work, world: int):
    """Rank of each field for a multi-GPU batched curvature run: whole fields,
    largest first, each to the rank with the least work so far (the longest-
    processing-time rule; ties to the lower rank), so every rank computes the
    same assignment from the same per-field work (interface-cell counts) and
    no field is split.  Returns a list of ranks, one per field."""
    order = sorted(range(len(work)), key=lambda i: (-int(work[i]), i))
    load = [0] * world
    owner = [0] * len(work)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(work[i])
    return owner


def barrier():
    if dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar (the slowest rank's time)."""
    if not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, world: int, steps: int, seconds_max: float) -> float:
    """Whole-job throughput: all units of all ranks over the slowest rank's time."""
    return units_per_rank * world * steps / seconds_max
