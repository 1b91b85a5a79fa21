"""Sharding and aggregation for multi-GPU runs (one process per GPU).

The likelihood calls of a sampler are independent (the paper's proposal
pool, Sec. III.B "CPU acceleration"), and the joint covariance of disjoint
segments and detectors is block-diagonal (Sec. II.B items 1 and 3): work
shards across ranks with no collective on the data path.  Ranks exchange
only timings and counts at the end (a max and a sum over ranks).
"""
from __future__ import annotations


def shard_columns(K: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [start, stop) of K residual columns for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(K, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_segments(work: list[float], world: int) -> list[list[int]]:
    """Assign segments (given their work, e.g. N'^2 K) to ranks: longest
    first to the least-loaded rank.  Deterministic for equal inputs."""
    loads = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(work)), key=lambda j: (-work[j], j)):
        r = min(range(world), key=lambda q: (loads[q], q))
        out[r].append(i)
        loads[r] += work[i]
    return [sorted(x) for x in out]


def aggregate(elapsed_s: float, evals: int, device=None) -> tuple[float, int]:
    """(max over ranks of elapsed seconds, sum over ranks of evaluations)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return elapsed_s, evals
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    n = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())
