"""GPU linearized Bregman (rska_linearized_bregman, the eta -> infinity limit
of eq. rska run as one full sweep of the row-split kernel per iteration)
against the oracle's FP64 iteration z <- z - step A^T (A x - b).

Bar: z and x within 1e-4 relative of the oracle after K iterations; the RSKA
counter and index sequence untouched, and RSKA continues from the linearized
Bregman iterate.
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
    from paper_2203_10838_gb300.rska import Solver
    return torch, oracle, Solver


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("m,n,s,lam,K", [
    (300, 1001, 20, 0.3, 40),      # one CTA (small sweep), n not a multiple of 4
    (3000, 2050, 30, 1.0, 30),     # about 20 rows per CTA per sweep
    (8000, 6000, 80, 2.0, 5),      # 53 rows per CTA per sweep
])
def test_linearized_bregman_parity(env, m, n, s, lam, K):
    torch, orc, Solver = env
    p = gaussian_problem(m, n, s, seed=m + n, noise=0.01)
    A = np.ascontiguousarray(p.A[:, :n])
    step = 1.0 / orc.sigma_max2(A)
    with Solver(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), lam, 8, 1.0, 0,
                n=n) as sol:
        sol.linearized_bregman(K, step)
        x, z = [v.cpu().numpy().astype(np.float64) for v in sol.get_x()]
    zr = orc.linearized_bregman(A, p.b.astype(np.float64), lam, step, K)
    assert rel(z, zr) <= REL_TOL, rel(z, zr)
    assert rel(x, orc.soft_shrink(zr, lam)) <= REL_TOL


def test_rska_continues_from_the_linearized_bregman_iterate(env):
    torch, orc, Solver = env
    p = gaussian_problem(1200, 700, 15, seed=99)
    A = np.ascontiguousarray(p.A[:, :700])
    step = 1.0 / orc.sigma_max2(A)
    b64 = p.b.astype(np.float64)
    with Solver(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.b).cuda(), 0.4, 16, 2.0, 3,
                n=700) as sol:
        sol.linearized_bregman(10, step)
        sol.solve(40)
        x = sol.get_x()[0].cpu().numpy().astype(np.float64)
        tau_g = sol.get_indices(0, 40).cpu().numpy()
    nu = orc.row_norms(A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=3, eta=16, k0=0, K=40)
    np.testing.assert_array_equal(tau_g, tau)
    z0 = orc.linearized_bregman(A, b64, 0.4, step, 10)
    zr = orc.rska_fixed(A, b64, 0.4, 2.0, 16, tau, z0=z0, nu=nu)
    assert rel(x, orc.soft_shrink(zr, 0.4)) <= REL_TOL
