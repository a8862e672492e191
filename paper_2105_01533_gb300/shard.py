"""Sharding of independent circuits across ranks (one process per GPU).

Circuits are independent, so the batched workload shards with no exchange on
the data path: every rank runs its own share and only the per-rank totals
(updates, elapsed time) are reduced for reporting. Shares are chosen by the
longest-processing-time rule on an estimate of each circuit's work.
"""

from __future__ import annotations

import heapq
from typing import List, Sequence

import numpy as np

from . import workloads as W


def circuit_work(c) -> int:
    """Work estimate of a batched circuit: gates x the nonzero bound
    min(cap, 2^(#branching gates)), the bound reached after its H gates."""
    g = c.gates
    nb = int(np.isin(g["op"], W.BRANCH_OPS).sum())
    return int(len(g)) * int(min(c.cap, 1 << min(nb, 40)))


def lpt_partition(works: Sequence[int], nranks: int) -> List[List[int]]:
    """Indices per rank: largest work first, each to the least-loaded rank
    (ties to the lowest rank). Deterministic."""
    if nranks < 1:
        raise ValueError("nranks >= 1")
    order = sorted(range(len(works)), key=lambda i: (-works[i], i))
    heap = [(0, r) for r in range(nranks)]
    parts: List[List[int]] = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + works[i], r))
    for p in parts:
        p.sort()
    return parts


def my_share(circuits, rank: int, world: int):
    parts = lpt_partition([circuit_work(c) for c in circuits], world)
    return [circuits[i] for i in parts[rank]]


def reduce_totals(updates: float, seconds: float, group=None):
    """(sum of updates, max of seconds) over ranks; plain values when not
    distributed. Only these two numbers cross ranks."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return updates, seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([updates, -seconds], dtype=torch.float64, device=dev)
    s = torch.tensor([updates], dtype=torch.float64, device=dev)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(s.item()), float(-t[1].item())
