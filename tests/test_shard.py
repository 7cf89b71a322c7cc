"""Multi-process (gloo, world size 2, CPU) coverage of the sharded path: the
partition helpers give every rank a disjoint share that together covers all
work, every rank computes the same partition independently, and the timing
that bench.py reports is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

from paper_2203_10838_gb300.shard import problem_shards, problem_work, rhs_shards
from synth import batched_sizes


def test_problem_shards_cover_and_balance():
    ms, ns = batched_sizes(4096, seed=2024, m_lo=200, m_hi=4000)
    for world in (1, 2, 3, 8):
        sh = problem_shards(ms, ns, 32, world)
        allp = np.concatenate([np.array(s, dtype=np.int64) for s in sh])
        assert np.array_equal(np.sort(allp), np.arange(4096))
        loads = [sum(problem_work(ms[p], ns[p], 32) for p in s) for s in sh]
        big = max(problem_work(m, n, 32) for m, n in zip(ms, ns))
        # LPT: the spread of the loads is at most the largest single job
        assert max(loads) - min(loads) <= big + 1e-6


def test_rhs_shards():
    for R, world in [(512, 1), (512, 2), (512, 3), (7, 4), (3, 5)]:
        sh = rhs_shards(R, world)
        assert sh[0][0] == 0 and sh[-1][1] == R
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        sizes = [b - a for a, b in sh]
        assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2203_10838_gb300.shard import max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, ns = batched_sizes(512, seed=7)
    mine = problem_shards(ms, ns, 32, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = max_over_ranks(10.0 + rank)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, gathered, t))


def test_two_gloo_ranks_agree_on_partition_and_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    g0, g1 = res[0][1], res[1][1]
    assert g0 == g1                       # both ranks computed the same partition
    allp = sorted(g0[0] + g0[1])
    assert allp == list(range(512))       # disjoint and complete
    assert res[0][2] == res[1][2] == 11.0  # the slowest rank's time
