"""Multi-GPU placement of independent simulations (one process per GPU).

The batched parameter sweep is a set of independent simulations: it shards
with no exchange on the data path.  Simulations are assigned to ranks by
the greedy longest-processing-time rule (largest agent count first, to the
least loaded rank), which keeps the most loaded rank within 4/3 of the
optimum.  A single-domain workload does not shard here: every rank steps
its own replica (the halo exchange of a domain decomposition is not part of
this library).  Timing and counters are combined on the host after the
timed region (max of times, sum of agent-updates).
"""
from __future__ import annotations

import heapq


def lpt_partition(sizes, n_ranks: int) -> list[list[int]]:
    """Indices of `sizes` per rank, largest first to the least loaded rank;
    ties go to the lower rank, so every rank computes the same partition."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(n_ranks)]
    heapq.heapify(heap)
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(p) for p in parts]


def shard(items, sizes, rank: int, world: int):
    """(global indices, items) of this rank's share of independent items."""
    idx = lpt_partition(sizes, world)[rank]
    return idx, [items[i] for i in idx]
