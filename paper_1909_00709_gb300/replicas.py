"""Host logic of running the path on several GPUs, one process per GPU.

The path shards without any exchange on the data path: every grid (and every grid of
a batch) is an independent unit, so ranks take disjoint sets of units and only the
timing is combined.  ``assign_grids`` splits a batch of uneven grids across ranks by
the longest-processing-time rule (largest grid first, to the least-loaded rank), which
bounds the slowest rank's share by 4/3 of the optimum; ``slowest`` and ``total``
combine per-rank numbers with one collective each (any torch.distributed backend:
NCCL on GPUs, gloo on CPUs in the tests).
"""
from __future__ import annotations

import heapq


def assign_grids(shapes, world: int):
    """Indices of `shapes` ((nx, ny, nz) each) per rank, balanced by point count."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(shapes)), key=lambda i: (-shapes[i][0] * shapes[i][1] * shapes[i][2], i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        nx, ny, nz = shapes[i]
        heapq.heappush(heap, (load + nx * ny * nz, r))
    return [sorted(v) for v in out]


def _reduce(value: float, op, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def slowest(ms: float, device=None) -> float:
    """The largest of the ranks' values (a job takes as long as its slowest rank)."""
    import torch.distributed as dist
    return _reduce(ms, dist.ReduceOp.MAX, device)


def total(count: float, device=None) -> float:
    """The sum of the ranks' values (work done by the whole job)."""
    import torch.distributed as dist
    return _reduce(count, dist.ReduceOp.SUM, device)
