"""Sharding of independent lattices (or serving requests) across ranks.

One process drives one GPU.  Independent lattices need no data exchange
between ranks, so a multi-GPU run is each rank advancing its own share of
the lattices; the only collectives are host-side: the max of the timed
region over ranks (the job is as slow as its slowest rank) and sums of
counters.  Works with any ``torch.distributed`` backend (``gloo`` on CPU
tensors, ``nccl`` on CUDA tensors).
"""
from __future__ import annotations

import heapq
import math


def assign(cells, world: int) -> list[list[int]]:
    """Greedy largest-first assignment of items (given by their cell
    counts) to ``world`` ranks, each item to the currently least-loaded rank
    (ties: lowest rank).  Deterministic: every rank computes the same answer
    from the same list.  Returns, per rank, its item indices in ascending
    order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(cells[i]), r))
    return [sorted(x) for x in out]


def my_items(cells, rank: int, world: int) -> list[int]:
    """The item indices rank ``rank`` of ``world`` owns."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return assign(cells, world)[rank]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def _tensor(values, device):
    import torch
    return torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)


def reduce_max(values, device="cpu"):
    """Element-wise max over ranks of a list of floats (identity without a
    process group)."""
    dist = _dist()
    if dist is None:
        return [float(v) for v in values]
    t = _tensor(values, device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def reduce_sum(values, device="cpu"):
    """Element-wise sum over ranks of a list of floats."""
    dist = _dist()
    if dist is None:
        return [float(v) for v in values]
    t = _tensor(values, device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()]


def gather(obj) -> list:
    """Every rank's ``obj`` (picklable), in rank order, on every rank."""
    dist = _dist()
    if dist is None:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def nearest_rank(sorted_values, q: float) -> float:
    """Nearest-rank percentile (q in (0, 1]) of an ascending list; 0 when
    empty (the definition the request server uses for its p50/p99)."""
    n = len(sorted_values)
    if n == 0:
        return 0.0
    k = min(n, max(1, math.ceil(q * n)))
    return float(sorted_values[k - 1])


def merged_sorted(values) -> list:
    """Every rank's values (e.g. per-request latencies), merged and sorted,
    on every rank."""
    return sorted(float(v) for part in gather(list(values)) for v in part)
