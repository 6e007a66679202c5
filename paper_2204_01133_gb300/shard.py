"""Multi-rank helpers: one process per GPU, no data-path collective.

The hot path shards by independent units: replicas of a single problem
(each rank runs its own instance, with its own Philox counter word), or the
instances of a batch split over the ranks.  Neither needs an exchange while
it runs; the only collectives are around the timed region (a barrier and the
maximum of the per-rank times).  Splitting one large domain over GPUs would
add a neighbour put of each rank's edge windows per step; on one-GPU machines
that remains a design (see the repository's design notes).
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
