"""Multi-GPU layout: one process per GPU, no collective on the data path.

A single all-pairs minimax-path solve (Algorithm 4 over one graph) does not
shard: its Boruvka rounds, leaf order and fill all read the whole matrix, and
one n = 65536 matrix pair fits one GPU's HBM many times over.  With N GPUs the
single-solve workload therefore runs as N independent replicas.  A batch of
independent graphs does shard: each rank solves a disjoint subset of the
graphs (weak scaling), and ranks only meet at the timing barrier and the
max-over-ranks reduction of the elapsed time.

The helpers here are host logic only (they run on the gloo backend in the CPU
tests) and work with or without an initialised process group.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def shard_graphs(sizes: Sequence[int], world: int) -> list[list[int]]:
    """Partition graph indices over `world` ranks, balancing the n^2 work.

    Longest-processing-time greedy: graphs in order of decreasing n^2 (ties by
    index) go to the rank with the least work so far (ties by rank).  The
    result is deterministic, so every rank computes the same partition without
    communicating.  Each rank's list is in increasing index order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda g: (-int(sizes[g]) ** 2, g))
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for g in order:
        load, r = heapq.heappop(heap)
        out[r].append(g)
        heapq.heappush(heap, (load + int(sizes[g]) ** 2, r))
    return [sorted(x) for x in out]


def rank_graphs(sizes: Sequence[int], rank: int, world: int) -> list[int]:
    """The graphs this rank solves (see shard_graphs)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return shard_graphs(sizes, world)[rank]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def barrier() -> None:
    d = _dist()
    if d is not None and d.get_world_size() > 1:
        d.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    d = _dist()
    if d is None or d.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """The sum of x over all ranks (x itself without a process group)."""
    d = _dist()
    if d is None or d.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t.item())
