"""Host-side logic of runs on several GPUs, one process per GPU.

Independent lattices never exchange data, so a run on N GPUs is either N
replicas of one lattice (each rank steps its own copy; "weak" scaling) or
a batch of independent flames split across the ranks.  Neither needs a
collective on the data path: the only collectives are the barrier around
the timed region and the maximum of the per-rank times, as the whole job
is as slow as its slowest rank.
"""
from __future__ import annotations

from typing import List, Sequence


def shard_lengths(lengths: Sequence[int], world: int) -> List[List[int]]:
    """Flame indices per rank, balancing the node counts: longest flame
    first onto the least-loaded rank (ties to the lowest rank), each rank's
    list in ascending index order.  Every flame lands on exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(lengths)), key=lambda i: (-int(lengths[i]), i)):
        r = min(range(world), key=lambda j: (load[j], j))
        out[r].append(k)
        load[r] += int(lengths[k])
    return [sorted(v) for v in out]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the value itself without a process
    group).  device: where the reduction tensor lives ("cuda" for NCCL,
    "cpu" for gloo)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: Sequence[int], steps: int, ms_max: float) -> float:
    """Lattice updates of all ranks per second of the slowest rank, in
    millions."""
    return float(sum(nodes_per_rank)) * steps / (ms_max * 1e-3) / 1e6
