"""Multi-rank helpers: one process per GPU.

Replicas and batches shard by independent units: each rank runs its own
instance (with its own Philox counter word), or a share of a batch's
instances split by work (longest processing time first).  Neither needs an
exchange while it runs; the only collectives are around the timed region (a
barrier and the maximum of the per-rank times).  Splitting one domain over
ranks by PE ranges, with the edge windows of every stage exchanged between
neighbouring ranks, is in ``rangesplit``.
"""
from __future__ import annotations

import heapq
import os


def env():
    """(rank, world size, local rank) from the torchrun environment."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def lpt_partition(costs, world: int):
    """Split unit indices over `world` ranks, largest cost first onto the
    least-loaded rank (longest-processing-time rule).  Returns one sorted
    index list per rank; together they cover every unit exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def max_over_ranks(value: float) -> float:
    """The maximum of a per-rank float over the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
