"""GPU estimate of sigma_max(A)^2 and alpha^*(eta) (rska_sigma_max2,
Corollary 1) against the oracle's eigenvalue of A^T A in FP64.

Bar: with a gap between the two largest singular values (a planted spike) the
Rayleigh quotient matches sigma_max^2 to 1e-5 after 60 iterations; on a plain
Gaussian matrix (top of the spectrum packed near the Marchenko-Pastur edge) it
stays a lower estimate within 3% after 100 iterations; ||A||_F^2 equals the
sum of the oracle's row norms and alpha^* follows Corollary 1 from the
returned values.
"""
import numpy as np
import pytest

from synth import gaussian_problem

pytestmark = pytest.mark.gpu


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


def estimate(env, A, eta, iters, seed=0):
    torch, orc, Solver = env
    m, n = A.shape
    b = np.ones(m, np.float32)
    with Solver(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), 0.5, eta, 1.0, 0,
                n=n) as sol:
        return sol.sigma_max2(iters, seed)


def test_spiked_matrix_converges(env):
    torch, orc, Solver = env
    rng = np.random.default_rng(3)
    m, n = 1500, 700
    x, y = rng.standard_normal(m), rng.standard_normal(n)
    A = (rng.standard_normal((m, n)) + 0.2 * np.outer(x, y)).astype(np.float32)
    s2, f2, al = estimate(env, A, 64, 60)
    exact = orc.sigma_max2(A)
    assert abs(s2 - exact) / exact <= 1e-5, (s2, exact)
    nu = orc.row_norms(A)
    np.testing.assert_allclose(f2, nu.sum(), rtol=1e-12)
    np.testing.assert_allclose(al, orc.alpha_star(64, s2, f2), rtol=1e-14)
    np.testing.assert_allclose(al, orc.alpha_star(64, exact, nu.sum()), rtol=1e-4)


def test_gaussian_matrix_lower_estimate(env):
    torch, orc, Solver = env
    p = gaussian_problem(3000, 1500, 20, seed=11)
    A = np.ascontiguousarray(p.A[:, :1500])
    s2, f2, al = estimate(env, A, 256, 100, seed=5)
    exact = orc.sigma_max2(A)
    assert exact * 0.97 <= s2 <= exact * (1 + 1e-5), (s2, exact)


def test_rank_one_gives_alpha_one(env):
    rng = np.random.default_rng(4)
    A = np.outer(rng.standard_normal(400), rng.standard_normal(300)).astype(np.float32)
    s2, f2, al = estimate(env, A, 128, 10)
    np.testing.assert_allclose(s2, f2, rtol=1e-5)
    np.testing.assert_allclose(al, 1.0, rtol=1e-3)
