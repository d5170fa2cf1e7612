"""Event sharding over GPUs: one process per GPU, events independent.

Events are the unit of work (the paper processes each event on its own), so
a multi-GPU run partitions the event list and needs no exchange in the data
path; the only collective is a host-side gather of per-event results to one
rank.  Partitioning is longest-processing-time first: events in decreasing
cost (hits, the vote's work driver) go one by one to the least-loaded rank,
which keeps every rank within one event's cost of the others.
"""
import heapq

import numpy as np


def partition(costs, world):
    """Indices of the events each rank processes (LPT greedy).

    costs: per-event cost (hit counts).  Returns a list of `world` sorted
    index arrays covering every event once.  Ties go to the lower rank and
    the lower event index, so every rank computes the same partition."""
    costs = np.asarray(costs, np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(costs.shape[0]), key=lambda e: (-int(costs[e]), e))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for e in order:
        load, r = heapq.heappop(heap)
        parts[r].append(e)
        heapq.heappush(heap, (load + int(costs[e]), r))
    return [np.array(sorted(p), np.int64) for p in parts]


def loads(costs, parts):
    costs = np.asarray(costs, np.int64)
    return [int(costs[p].sum()) for p in parts]


def gather_results(local, dst=0, group=None):
    """Gather {event index: result} dicts from every rank to rank dst.

    Uses torch.distributed's object gather (works on gloo and nccl process
    groups; with nccl the current CUDA device carries the bytes).  Returns
    the merged dict on dst and None elsewhere.  Without an initialised
    process group the local dict is returned as is."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return dict(local)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    out = [None] * world if rank == dst else None
    dist.gather_object(local, out, dst=dst, group=group)
    if rank != dst:
        return None
    merged = {}
    for part in out:
        dup = merged.keys() & part.keys()
        if dup:
            raise RuntimeError(f"events {sorted(dup)[:5]} processed by two ranks")
        merged.update(part)
    return merged
