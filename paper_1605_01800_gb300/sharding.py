"""Host-side sharding of a batch of independent lattices across ranks.

The lattices of a batch never exchange data, so several GPUs split a batch
with no collective on the data path: each rank creates a context over its own
share and steps it. Shares are balanced by node count with the
longest-processing-time rule (largest lattice first, to the least-loaded rank,
ties to the lowest rank), which every rank computes identically from the
lattice sizes alone.
"""
from typing import List, Sequence


def lpt_partition(sizes: Sequence[int], n_ranks: int) -> List[List[int]]:
    """Indices of `sizes` assigned to each of `n_ranks` ranks, each list in
    ascending index order."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * n_ranks
    parts: List[List[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(p) for p in parts]


def shard(specs: Sequence, rank: int, world: int) -> list:
    """The lattices (e.g. ``inputs.LatticeSpec``) rank `rank` of `world` owns."""
    parts = lpt_partition([s.nx * s.ny for s in specs], world)
    return [specs[i] for i in parts[rank]]
