"""Host-side logic for running on several GPUs of one node: one process per GPU.

Events are independent (the method has no coupling between them), so the work shards without a
data-path collective: every rank advances its own events, and the process group is used only for
a barrier and for reducing timings.  A batch of events of uneven sizes is partitioned across
ranks by cell count, largest event first onto the least-loaded rank.
"""
from __future__ import annotations

import os


def shard_events(cells: list[int], world: int) -> list[list[int]]:
    """Partition event indices over `world` ranks: events in decreasing cell count (ties by
    index), each onto the rank with the fewest cells so far (ties by rank).  Deterministic; every
    rank computes the same answer.  Returns the sorted event indices of every rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    shards: list[list[int]] = [[] for _ in range(world)]
    for ev in sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(ev)
        load[r] += int(cells[ev])
    return [sorted(s) for s in shards]


def rank_share(cells: list[int], world: int, rank: int) -> tuple[list[int], int]:
    """This rank's events of one batch (shard_events) and the batch's total cell count: every rank
    advances only its own share, in one context, with no data-path collective."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return shard_events(cells, world)[rank], int(sum(int(c) for c in cells))


def env_ranks() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> tuple[int, int, int]:
    """Join the process group when launched with more than one rank."""
    world, rank, local = env_ranks()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    """The sum over all ranks (e.g. cells advanced by the whole job)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
