"""GPU parity of the batched solver (rska_batch_*, one persistent launch over
many independent problems) against the FP64 oracle run problem by problem
with the same index contract (counter word 3 = problem id).

Bar: row norms, alias tables bit-exact; after a fixed K every problem's
iterate within 1e-4 relative of the oracle's; with the residual stopping rule,
every problem that reports convergence really has ||A x - b|| / ||b|| <= tol
(checked by the oracle on the GPU's iterate) and stopped on a check point.
"""
import numpy as np
import pytest

from synth import batched_sizes, gaussian_problem, pack_batch

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10838_gb300 import build
    build.build()
    import oracle
    oracle.build()
    from paper_2203_10838_gb300.rska import BatchSolver
    return torch, oracle, BatchSolver


def make_batch(shapes, seed0):
    probs = []
    for i, (m, n) in enumerate(shapes):
        probs.append(gaussian_problem(m, n, max(1, n // 20), seed=seed0 + i))
    return probs


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


SHAPES = [(8, 8), (37, 13), (200, 96), (64, 200), (300, 150), (600, 296), (45, 45), (120, 61),
          (500, 252), (16, 4), (1000, 504), (333, 2001), (90, 40), (2, 3), (700, 350), (250, 128)]


def test_batched_parity_fixed_iterations(env):
    torch, orc, BatchSolver = env
    probs = make_batch(SHAPES, 3000)
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    lam, eta, t, seed, K = 0.5, 32, 1.0, 99, 60  # t = 1 is admissible for every shape here
    Ad = torch.from_numpy(A).cuda()
    bd = torch.from_numpy(b).cuda()
    with BatchSolver(Ad, bd, a_off, m, n, lda, b_off, lam, eta, t, seed) as bs:
        nu_g, thr_g, al_g = [v.cpu().numpy() for v in bs.get_tables()]
        bs.solve(K, tol=0.0)
        iters, rr = bs.results()
        x, z = [v.cpu().numpy().astype(np.float64) for v in bs.get_x()]
        xo = bs.x_off
    assert np.all(iters == K)
    ro = 0
    for p, pr in enumerate(probs):
        Ap = pr.A[:, :pr.n]
        nu = orc.row_norms(Ap)
        thr, alias = orc.alias_build(nu)
        np.testing.assert_array_equal(nu_g[ro:ro + pr.m], nu)
        np.testing.assert_array_equal(thr_g[ro:ro + pr.m].view(np.uint32), thr)
        np.testing.assert_array_equal(al_g[ro:ro + pr.m], alias)
        ro += pr.m
        zr = orc.rska(Ap, pr.b.astype(np.float64), lam, eta, t, seed, K, problem=p,
                      tables=(nu, thr, alias))
        xr = orc.soft_shrink(zr, lam)
        zg = z[xo[p]:xo[p] + pr.n]
        xg = x[xo[p]:xo[p] + pr.n]
        assert rel(zg, zr) <= REL_TOL, (p, pr.m, pr.n, rel(zg, zr))
        if np.linalg.norm(xr) > 0:
            assert rel(xg, xr) <= REL_TOL, (p, pr.m, pr.n, rel(xg, xr))
        else:
            assert np.all(xg == 0)
        rr_o, _ = orc.metrics(Ap, pr.b.astype(np.float64), zg, lam)
        assert abs(rr[p] - rr_o) <= 1e-5 * max(rr_o, 1e-12) + 1e-12, (p, rr[p], rr_o)


def test_batched_stopping_rule(env):
    """m log-uniform in [200, 1200], n = m/2 (multiple of 8), lambda = 1,
    eta = 32, t = 16: every problem stops at a check point with a relative
    residual <= 1e-6."""
    torch, orc, BatchSolver = env
    ms, ns = batched_sizes(40, seed=5, m_lo=200, m_hi=1200)
    probs = make_batch(list(zip(ms, ns)), 4000)
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    tol = 1e-6
    with BatchSolver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), a_off, m, n, lda,
                     b_off, 1.0, 32, 16.0, 7) as bs:
        bs.solve(200000, tol=tol)
        iters, rr = bs.results()
        x, z = [v.cpu().numpy().astype(np.float64) for v in bs.get_x()]
        xo = bs.x_off
    for p, pr in enumerate(probs):
        C = -(-pr.m // 32)
        assert 0 < iters[p] < 200000 and iters[p] % C == 0, (p, iters[p], C)
        assert rr[p] <= tol
        rr_o, _ = orc.metrics(pr.A[:, :pr.n], pr.b.astype(np.float64),
                              z[xo[p]:xo[p] + pr.n], 1.0)
        assert rr_o <= tol * 1.001, (p, rr[p], rr_o)


def test_batched_rejects_bad_problems(env):
    torch, orc, BatchSolver = env
    from paper_2203_10838_gb300._lib import RSKAError
    probs = make_batch([(20, 8), (30, 12)], 50)
    probs[1].A[5] = 0.0
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    with pytest.raises(RSKAError) as e:
        BatchSolver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), a_off, m, n, lda,
                    b_off, 1.0, 8, 4.0, 1)
    assert e.value.code == 2
    probs = make_batch([(20, 3000)], 51)
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    with pytest.raises(RSKAError) as e:
        BatchSolver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), a_off, m, n, lda,
                    b_off, 1.0, 8, 4.0, 1)
    assert e.value.code == 7


def test_batched_limits(env):
    """n = 2688 (the largest row a warp keeps in registers) and eta = 448 (the
    most rows of one iteration the index ring holds), with small and ragged
    problems in the same launch."""
    torch, orc, BatchSolver = env
    probs = make_batch([(3000, 2688), (500, 2688), (449, 17), (900, 450), (5, 3)], 6000)
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    lam, eta, t, seed, K = 0.5, 448, 1.0, 3, 15  # t = 1 is admissible for every shape
    with BatchSolver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), a_off, m, n, lda,
                     b_off, lam, eta, t, seed) as bs:
        bs.solve(K, tol=0.0)
        iters, rr = bs.results()
        x, z = [v.cpu().numpy().astype(np.float64) for v in bs.get_x()]
        xo = bs.x_off
    assert np.all(iters == K)
    for p, pr in enumerate(probs):
        Ap = pr.A[:, :pr.n]
        zr = orc.rska(Ap, pr.b.astype(np.float64), lam, eta, t, seed, K, problem=p)
        assert rel(z[xo[p]:xo[p] + pr.n], zr) <= REL_TOL, (p, pr.m, pr.n)


def test_batched_full_configuration_sampled(env):
    """The benchmark's 4096 systems (m log-uniform in [200, 4000], n = m/2,
    s = n/20, lambda = 1, eta = 32, t = 16) in one launch for a fixed 40
    iterations; a seeded subset of 64 problems, the eight largest among them,
    checked against the FP64 oracle."""
    torch, orc, BatchSolver = env
    from synth import batched_problem_set
    A, a_off, m, n, lda, b, b_off, _ = batched_problem_set(4096, seed=2024)
    lam, eta, t, seed, K = 1.0, 32, 16.0, 11, 40
    with BatchSolver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), a_off, m, n, lda,
                     b_off, lam, eta, t, seed) as bs:
        bs.solve(K, tol=0.0)
        iters, rr = bs.results()
        x, z = [v.cpu().numpy().astype(np.float64) for v in bs.get_x()]
        xo = bs.x_off
    assert np.all(iters == K)
    order = np.argsort(np.asarray(m) * np.asarray(n))
    largest = [int(p) for p in order[-8:]]
    rest = np.setdiff1d(np.arange(4096), largest)
    check = largest + [int(p) for p in np.random.default_rng(64).choice(rest, 56, replace=False)]
    assert len(set(check)) == 64
    for p in check:
        mp, np_, lp = int(m[p]), int(n[p]), int(lda[p])
        Ap = A[int(a_off[p]):int(a_off[p]) + mp * lp].reshape(mp, lp)[:, :np_]
        bp = b[int(b_off[p]):int(b_off[p]) + mp].astype(np.float64)
        zr = orc.rska(np.ascontiguousarray(Ap), bp, lam, eta, t, seed, K, problem=int(p))
        assert rel(z[xo[p]:xo[p] + np_], zr) <= REL_TOL, (p, mp, np_)


@pytest.mark.parametrize("shapes", [
    [(1, 1), (1, 9), (7, 1), (3, 2), (50, 30)],   # 1 x 1, one row, one column, tiny, ragged
    [(300, 150)],                                  # a batch of one problem
])
def test_batched_degenerate_shapes(env, shapes):
    torch, orc, BatchSolver = env
    probs = make_batch(shapes, 7000)
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    lam, eta, t, seed, K = 0.1, 5, 1.0, 23, 30
    with BatchSolver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), a_off, m, n, lda,
                     b_off, lam, eta, t, seed) as bs:
        bs.solve(K, tol=0.0)
        iters, rr = bs.results()
        z = bs.get_x()[1].cpu().numpy().astype(np.float64)
        xo = bs.x_off
    assert np.all(iters == K)
    for p, pr in enumerate(probs):
        zr = orc.rska(pr.A[:, :pr.n], pr.b.astype(np.float64), lam, eta, t, seed, K, problem=p)
        assert rel(z[xo[p]:xo[p] + pr.n], zr) <= REL_TOL, (p, pr.m, pr.n)
