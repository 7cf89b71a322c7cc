"""Parameter admissibility of the configurations (Theorem th:RSKA with
W = t I): the rate needs s_max(T) < 1, where Lemma lm:svt gives
s_max(T) = (t / (2 eta)) (1 + (eta - 1) sigma_max(A)^2 / ||A||_F^2), i.e.
t < 2 alpha*(eta).  Checked with the exact sigma_max(A)^2 (FP64 eigenvalue)
on the seeded matrices the configurations use, where that is cheap: the
1000 x 500 system (t = 1 and t = alpha*), the eight batched problems with the
fewest rows (the largest sigma_max^2 / ||A||_F^2 of the 4096) and four of the
64 unrolled problems.
"""
import numpy as np
import pytest

from synth import batched_sizes, gaussian_problem


def s_max_T(orc, A, eta, t):
    A = np.ascontiguousarray(A, dtype=np.float32)
    s = orc.sigma_max2(A) / orc.row_norms(A).sum()
    return t / (2.0 * eta) * (1.0 + (eta - 1) * s)


def alpha_star_mp(m, n, eta):
    s2 = (np.sqrt(m) + np.sqrt(n)) ** 2
    return eta / (1.0 + (eta - 1) * s2 / (m * n))


@pytest.mark.parametrize("t", [1.0, float(alpha_star_mp(1000, 500, 10))])
def test_small_configuration(orc, t):
    p = gaussian_problem(1000, 500, 25, seed=1000)
    assert s_max_T(orc, p.A[:, :500], 10, t) < 1.0


def test_batched_configuration_smallest_problems(orc):
    seed, eta, t = 2024, 32, 16.0
    m, n = batched_sizes(4096, seed)
    for p in np.argsort(m, kind="stable")[:8]:
        mp, np_ = int(m[p]), int(n[p])
        pr = gaussian_problem(mp, np_, np_ // 20, seed=seed + 1 + int(p))
        v = s_max_T(orc, pr.A[:, :np_], eta, t)
        assert v < 1.0, (int(p), mp, np_, v)


def test_unrolled_configuration(orc):
    for i in range(4):
        pr = gaussian_problem(2048, 1024, 50, seed=700 + i, noise=0.01)
        assert s_max_T(orc, pr.A[:, :1024], 64, 32.0) < 1.0
