"""Host-side work partitioning for one process per GPU.

Every form of the path shards without a data-path collective: the batched
and unrolled forms are independent problems, the multi-RHS form has
independent right-hand sides that share A and the index stream (each rank
holds A and draws the same tau from the same seed).  Ranks only agree on the
timing (maximum over ranks) and, after the timed region, gather the
per-problem (or per-right-hand-side) results.  No device work happens here.
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


def gather_by_unit(mine, results, world: int):
    """Every rank's per-unit results gathered on every rank: a dict from unit
    index (problem or right-hand side) to its result.  `mine` lists this
    rank's units and `results` their results in the same order."""
    mine = [int(u) for u in mine]
    results = list(results)
    if len(mine) != len(results):
        raise ValueError("one result per unit")
    if world == 1:
        return dict(zip(mine, results))
    import torch.distributed as dist
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, results))
    out = {}
    for units, res in gathered:
        for u, r in zip(units, res):
            if u in out:
                raise RuntimeError(f"unit {u} solved on two ranks")
            out[u] = r
    return out


def sharded_run(shards, solve, rank: int, world: int, device=None):
    """The rank loop of the sharded batched and multi-RHS forms: this rank
    solves its share `shards[rank]` (a list of unit indices) with
    `solve(units) -> (results, seconds)`, results in the order of `units` and
    seconds the rank's timed solve; then the slowest rank's time is agreed
    (maximum over ranks) and the results of every rank are gathered.
    Returns (results by unit index, this rank's seconds, slowest seconds)."""
    mine = list(shards[rank])
    results, seconds = solve(mine)
    slowest = max_over_ranks(seconds, device)
    return gather_by_unit(mine, results, world), float(seconds), slowest
