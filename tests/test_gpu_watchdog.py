"""Device-side watchdog of the persistent kernels (failure detection without a
GPU fault).

Every wait inside the solver kernels (the grid barrier, the mbarrier ring of
the row-split kernel, the tensor-core pipeline of the multi-right-hand-side
form) gives up after a limit set per context (rska_set_option(ctx, 1, us),
rska_mrhs_set_option(h, 2, us)).  With a limit of zero the first wait that is
not satisfied at its first poll runs out (every grid barrier has a CTA that
arrives first and must wait): the kernel records RSKA_ETIMEOUT in the
context's status word, lets the copies it has already issued land, and
returns.  Nothing hangs: the
waits give up and return, and copies in flight are always drained.

Checked: the next synchronizing call reports RSKA_ETIMEOUT, the error is
sticky, and after rska_reset with the default limit restored the same context
solves the problem as the FP64 oracle does (indices bit-exact, iterate within
1e-4).
"""
import numpy as np
import pytest

from synth import gaussian_problem, multi_rhs_problem

pytestmark = pytest.mark.gpu

ETIMEOUT = 6
DEFAULT_LIMIT_US = 2_000_000


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10838_gb300 import build
    build.build()
    import oracle
    oracle.build()
    return torch, oracle


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_small_system_kernel_wait_limit_runs_out_and_context_recovers(env):
    """The one-CTA small-system kernel has no grid barrier; its waits are the
    ring's: the consumers' wait for a slot's rows and the producer's wait for
    a released slot, each probed once without blocking before it spins.
    With a zero limit the first wait whose phase is not complete at that
    probe runs out (the consumers reach their first wait while the first
    rows are still being fetched; and whichever side is faster waits for the
    other within a few iterations), the kernel records ETIMEOUT, drains the
    copies it issued and returns; after rska_reset the context solves as the
    oracle does.  The expiry depends on timing, so up to five launches of
    2000 iterations are given to show it."""
    torch, orc = env
    from paper_2203_10838_gb300._lib import RSKAError
    from paper_2203_10838_gb300.rska import KERNEL, Solver
    m, n, s, eta, lam, t, seed, K = 1000, 500, 25, 10, 1.0, 1.0, 3, 300
    prob = gaussian_problem(m, n, s, seed=901)
    A = torch.from_numpy(prob.A).cuda()
    b = torch.from_numpy(prob.b).cuda()
    with Solver(A, b, lam, eta, t, seed, n=n) as sol:
        sol.set_option("kernel", KERNEL["small"])
        sol.set_option("watchdog_us", 0)
        code = None
        for _ in range(5):
            sol.solve(2000)
            try:
                sol.get_x()
            except RSKAError as e:
                code = e.code
                break
            sol.reset()
        assert code == ETIMEOUT
        with pytest.raises(RSKAError) as ei:
            sol.solve(1)
        assert ei.value.code == ETIMEOUT
        sol.reset()
        sol.set_option("watchdog_us", DEFAULT_LIMIT_US)
        sol.solve(K)
        x, z = [v.cpu().numpy().astype(np.float64) for v in sol.get_x()]
        idx = sol.get_indices(0, K).cpu().numpy()
        assert sol.query("kernel") == KERNEL["small"]
    nu = orc.row_norms(prob.A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    np.testing.assert_array_equal(idx, tau)
    zr = orc.rska_fixed(prob.A, prob.b.astype(np.float64), lam, t, eta, tau, nu=nu)
    assert rel(z, zr) <= 1e-4
    assert rel(x, orc.soft_shrink(zr, lam)) <= 1e-4


@pytest.mark.parametrize("kernel", ["rows", "column"])
def test_single_system_wait_limit_runs_out_and_context_recovers(env, kernel):
    torch, orc = env
    from paper_2203_10838_gb300._lib import RSKAError
    from paper_2203_10838_gb300.rska import KERNEL, Solver
    m, n, s, eta, lam, t, seed, K = 4000, 2000, 40, 512, 1.0, 64.0, 3, 60
    prob = gaussian_problem(m, n, s, seed=900)
    A = torch.from_numpy(prob.A).cuda()
    b = torch.from_numpy(prob.b).cuda()
    with Solver(A, b, lam, eta, t, seed, n=n) as sol:
        sol.set_option("kernel", KERNEL[kernel])
        sol.set_option("watchdog_us", 0)
        sol.solve(200)
        with pytest.raises(RSKAError) as ei:
            sol.get_x()
        assert ei.value.code == ETIMEOUT
        # sticky until rska_reset
        with pytest.raises(RSKAError) as ei:
            sol.solve(1)
        assert ei.value.code == ETIMEOUT
        assert sol.query("grid") > 1
        sol.reset()
        sol.set_option("watchdog_us", DEFAULT_LIMIT_US)
        sol.solve(K)
        x, z = [v.cpu().numpy().astype(np.float64) for v in sol.get_x()]
        idx = sol.get_indices(0, K).cpu().numpy()
        assert sol.query("kernel") == KERNEL[kernel]
    An = prob.A[:, :n]
    nu = orc.row_norms(An)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    np.testing.assert_array_equal(idx, tau)
    zr = orc.rska_fixed(An, prob.b.astype(np.float64), lam, t, eta, tau, nu=nu)
    assert rel(z, zr) <= 1e-4
    assert rel(x, orc.soft_shrink(zr, lam)) <= 1e-4


@pytest.mark.parametrize("form", ["staged", "persistent"])
def test_multi_rhs_wait_limit_runs_out_and_context_recovers(env, form):
    torch, orc = env
    from paper_2203_10838_gb300._lib import RSKAError
    from paper_2203_10838_gb300.rska import MRHS_FORM, MultiRHS
    m, n, R, s, eta, lam, t, seed, K = 1024, 512, 64, 10, 128, 0.3, 8.0, 4, 20
    p = multi_rhs_problem(m, n, R, s, seed=31)
    A = torch.from_numpy(p.A16.view(np.int16)).cuda().view(torch.bfloat16)
    B = torch.from_numpy(p.B).cuda()
    with MultiRHS(A, B, lam, eta, t, seed, n=n) as h:
        h.set_option("form", MRHS_FORM[form])
        h.set_option("watchdog_us", 0)
        h.solve(70)
        with pytest.raises(RSKAError) as ei:
            h.get_x()
        assert ei.value.code == ETIMEOUT
        with pytest.raises(RSKAError) as ei:
            h.solve(1)
        assert ei.value.code == ETIMEOUT
        h.reset()
        h.set_option("watchdog_us", DEFAULT_LIMIT_US)
        h.solve(K)
        x, z = [v.cpu().numpy().astype(np.float64) for v in h.get_x()]
    A32 = np.ascontiguousarray(p.A[:, :n])
    nu = orc.row_norms(A32)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    rows = list(range(0, R, 7))
    Zr = orc.rska_mrhs(A32, p.B.astype(np.float64), lam, t, eta, tau, nu=nu, rows=rows)
    for r, j in enumerate(rows):
        assert rel(z[j], Zr[r]) <= 1e-4, (j, rel(z[j], Zr[r]))
