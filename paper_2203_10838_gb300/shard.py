"""Host-side work partitioning for one process per GPU.

Every form of the path shards without a data-path collective: the batched
and unrolled forms are independent problems, the multi-RHS form has
independent right-hand sides that share A and the index stream (each rank
holds A and draws the same tau from the same seed).  Ranks only agree on the
timing (maximum over ranks).  No device work happens here.
"""
from __future__ import annotations

import heapq


def problem_work(m: int, n: int, eta: int) -> float:
    """Estimated cost of one problem of the batched form: iterations grow
    about like n and each moves eta rows of n floats, plus one epoch per
    exact residual pass."""
    return float(n) * n + float(m) * n / max(1, eta)


def problem_shards(ms, ns, eta: int, world: int):
    """Longest-processing-time-first assignment of problems to `world` ranks:
    problems sorted by estimated work (ties by index), each given to the rank
    with the least work so far (ties by rank).  Returns one sorted index list
    per rank; together they cover every problem exactly once."""
    order = sorted(range(len(ms)), key=lambda p: (-problem_work(ms[p], ns[p], eta), p))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for p in order:
        load, r = heapq.heappop(heap)
        shards[r].append(p)
        heapq.heappush(heap, (load + problem_work(ms[p], ns[p], eta), r))
    return [sorted(s) for s in shards]


def rhs_shards(R: int, world: int):
    """Contiguous blocks of right-hand sides, sizes differing by at most one."""
    base, extra = divmod(R, world)
    out, start = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank scalar over the process group (the time of
    the slowest rank); the value itself when no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
