"""GPU parity of general row weights (rska_set_weights; eq. rska with W =
diag(w), Sec. 5 variants v3 and v4) against the FP64 oracle's weighted step.

Bar: row norms, the alias table (over nu for v3, over nu / w for v4) and every
sampled index bit-exact; iterates after K iterations within 1e-4 relative.
Weights are drawn from U[0, 1] (Sec. 5) plus 1e-3, as float32.
"""
import numpy as np
import pytest

from synth import gaussian_problem

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
    from paper_2203_10838_gb300.rska import KERNEL, Solver
    return torch, oracle, Solver, KERNEL


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def weights(m, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.0, 1.0, m) + 1e-3).astype(np.float32)


def run_weighted(env, m, n, s, eta, lam, t, seed, K, couple, kernel, grid=None, noise=0.0,
                 pseed=None):
    torch, orc, Solver, KERNEL = env
    prob = gaussian_problem(m, n, s, seed=pseed if pseed is not None else 2000 + seed,
                            noise=noise)
    w = weights(m, seed + 77)
    A = torch.from_numpy(prob.A).cuda()
    b = torch.from_numpy(prob.b).cuda()
    with Solver(A, b, lam, eta, t, seed, n=n) as sol:
        sol.set_option("kernel", KERNEL[kernel])
        if grid is not None:
            sol.set_option("grid", grid)
        sol.set_weights(torch.from_numpy(w).cuda(), couple=couple)
        nu_g, thr_g, alias_g = [v.cpu().numpy() for v in sol.get_tables()]
        sol.solve(K)
        x, z = [v.cpu().numpy().astype(np.float64) for v in sol.get_x()]
        idx = sol.get_indices(0, K).cpu().numpy()
        used = sol.query("kernel")
    An = prob.A[:, :n]
    nu = orc.row_norms(An)
    rho = nu / w.astype(np.float64) if couple else nu
    thr, alias = orc.alias_build(rho)
    np.testing.assert_array_equal(nu_g, nu)
    np.testing.assert_array_equal(thr_g.view(np.uint32), thr)
    np.testing.assert_array_equal(alias_g, alias)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    np.testing.assert_array_equal(idx, tau)
    zr = orc.rska_fixed(An, prob.b.astype(np.float64), lam, t, eta, tau, nu=nu,
                        w=w.astype(np.float64))
    xr = orc.soft_shrink(zr, lam)
    return rel(x, xr), rel(z, zr), used


@pytest.mark.parametrize("couple", [False, True])
def test_weighted_parity_small_system_kernel(env, couple):
    # 600 x 250 (the last float4 of a row is partly valid), eta = 12, on the
    # one-CTA kernel: the weights reach it through the per-row scale
    rx, rz, used = run_weighted(env, 600, 250, 10, 12, 0.5, 1.0, 3, 300, couple, "small")
    assert used == 3
    assert rx <= REL_TOL and rz <= REL_TOL, (couple, rx, rz)


@pytest.mark.parametrize("kernel", ["rows", "column"])
@pytest.mark.parametrize("couple", [False, True])
def test_weighted_parity(env, couple, kernel):
    # 1000 x 2050 (the last float4 of a row is partly valid), eta = 96 over 16 CTAs
    rx, rz, used = run_weighted(env, 1000, 2050, 30, 96, 0.5, 1.0, 3, 150, couple, kernel,
                                grid=16, noise=0.01)
    assert used == (2 if kernel == "rows" else 1)
    assert rx <= REL_TOL and rz <= REL_TOL, (couple, kernel, rx, rz)


def test_weighted_v4_full_size_configuration(env):
    """The benchmark's 20000 x 10000 system (1% noise, lambda = 2, eta = 1024)
    with v4 weights and t = 1 (the paper's v4 has no extra step), 30 iterations
    of the automatically chosen kernel."""
    rx, rz, used = run_weighted(env, 20000, 10000, 200, 1024, 2.0, 1.0, 0, 30, True, "auto",
                                noise=0.01, pseed=1001)
    assert rx <= REL_TOL and rz <= REL_TOL, (rx, rz, used)


def test_uniform_restore_and_invalid_weights(env):
    torch, orc, Solver, KERNEL = env
    from paper_2203_10838_gb300._lib import RSKAError
    prob = gaussian_problem(300, 200, 10, seed=17)
    A = torch.from_numpy(prob.A).cuda()
    b = torch.from_numpy(prob.b).cuda()
    with Solver(A, b, 0.3, 8, 1.0, 5, n=200) as sol:
        base = [v.cpu().numpy() for v in sol.get_tables()]
        w = weights(300, 9)
        sol.set_weights(torch.from_numpy(w).cuda(), couple=True)
        coupled = [v.cpu().numpy() for v in sol.get_tables()]
        assert not np.array_equal(coupled[1], base[1])
        for bad in (0.0, -1.0, np.nan, np.inf):
            wb = w.copy()
            wb[123] = bad
            with pytest.raises(RSKAError) as e:
                sol.set_weights(torch.from_numpy(wb).cuda(), couple=False)
            assert e.value.code == 1
            now = [v.cpu().numpy() for v in sol.get_tables()]
            for a, c in zip(now, coupled):
                np.testing.assert_array_equal(a, c)
        sol.set_weights(None)
        for a, c in zip([v.cpu().numpy() for v in sol.get_tables()], base):
            np.testing.assert_array_equal(a, c)
        # uniform weights again: the solve equals the unweighted oracle
        sol.solve(50)
        x = sol.get_x()[0].cpu().numpy().astype(np.float64)
    An = prob.A[:, :200]
    nu = orc.row_norms(An)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=5, eta=8, k0=0, K=50)
    xr = orc.soft_shrink(orc.rska_fixed(An, prob.b.astype(np.float64), 0.3, 1.0, 8, tau, nu=nu),
                         0.3)
    assert rel(x, xr) <= REL_TOL
