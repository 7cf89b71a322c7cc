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


# --------------------------------------------------------------------------
# The rank loop of the sharded batched and multi-RHS forms (shard.sharded_run)
# driven on two gloo ranks with a host stand-in for the GPU solve (the FP64
# oracle): the gathered per-problem and per-right-hand-side results must equal
# the unsharded run's, element by element.
# --------------------------------------------------------------------------
SH_P, SH_SEED, SH_ETA, SH_LAM, SH_T, SH_K, SH_RSEED = 12, 99, 4, 0.3, 2.0, 25, 5
SH_M, SH_N, SH_R = 40, 16, 10


def _batched_stand_in(units, orc):
    """Solve problems `units` of the sharded set on the host: each with its
    own data (generated for the subset only) and its index stream id = its
    index in the whole set, as the GPU batch gets with set_stream_ids."""
    from synth import batched_problem_set
    A, a_off, m, n, lda, b, b_off, _ = batched_problem_set(SH_P, SH_SEED, 20, 60, subset=units)
    out = []
    for j, p in enumerate(units):
        Ap = A[a_off[j]:a_off[j] + m[j] * lda[j]].reshape(m[j], lda[j])[:, :n[j]]
        bp = b[b_off[j]:b_off[j] + m[j]].astype(np.float64)
        out.append(orc.rska(Ap, bp, SH_LAM, SH_ETA, SH_T, SH_RSEED, SH_K, problem=p))
    return out


def _mrhs_stand_in(units, orc):
    """Right-hand sides `units` of one shared-A problem, solved with the index
    stream of problem 0 (shared by every rank)."""
    from synth import gaussian_problem
    pr = gaussian_problem(SH_M, SH_N, 3, seed=SH_SEED)
    A = pr.A[:, :SH_N]
    rng = np.random.default_rng(SH_SEED)
    B = rng.standard_normal((SH_R, SH_M))
    nu = orc.row_norms(A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=SH_RSEED, eta=SH_ETA, k0=0, K=SH_K)
    return list(orc.rska_mrhs(A, B[list(units)], SH_LAM, SH_T, SH_ETA, tau, nu=nu))


def _sharded_worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from paper_2203_10838_gb300.shard import sharded_run
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.build()
    ms, ns = batched_sizes(SH_P, SH_SEED, 20, 60)
    shards = problem_shards(ms, ns, SH_ETA, world)
    by_p, sec, slow = sharded_run(
        shards, lambda u: (_batched_stand_in(u, oracle), 1.0 + rank), rank, world)
    rshards = [list(range(a, b)) for a, b in rhs_shards(SH_R, world)]
    by_j, _, _ = sharded_run(rshards, lambda u: (_mrhs_stand_in(u, oracle), 0.5), rank, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, by_p, slow, by_j, shards[rank]))


def test_sharded_rank_loop_matches_the_unsharded_run(orc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    # both ranks hold every result; the ranks really split the work
    assert res[0][4] and res[1][4] and not set(res[0][4]) & set(res[1][4])
    whole_p = _batched_stand_in(list(range(SH_P)), orc)
    whole_j = _mrhs_stand_in(list(range(SH_R)), orc)
    for rank, by_p, slow, by_j, _ in res:
        assert slow == 2.0
        assert sorted(by_p) == list(range(SH_P)) and sorted(by_j) == list(range(SH_R))
        for p in range(SH_P):
            np.testing.assert_array_equal(by_p[p], whole_p[p])
        for j in range(SH_R):
            np.testing.assert_array_equal(by_j[j], whole_j[j])
