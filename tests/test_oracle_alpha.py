"""Pins for the oracle's sigma_max(A)^2 and alpha^*(eta) (Corollary 1, uniform
weights) against closed forms:

* rank one A = x y^T: sigma_max^2 = ||x||^2 ||y||^2 = ||A||_F^2, so alpha^* = 1
  for every eta (the averaged directions all coincide);
* orthogonal rows of equal norm c: sigma_max^2 = c^2 and ||A||_F^2 = m c^2,
  alpha^* = eta / (1 + (eta - 1)/m);
* a diagonal matrix: sigma_max^2 = max d_i^2;
* eta = 1 gives alpha^* = 1 (RSK, no averaging);
* alpha^* maximises the rate bound of Theorem th:RSKA with W = alpha I,
  L(alpha) = alpha - alpha/(2 eta) (alpha (eta - 1) s + alpha),
  s = sigma_max^2/||A||_F^2 (its derivative vanishes at alpha^*, and
  L(alpha^*) = alpha^*/2 as Corollary 1 states).
"""
import numpy as np
import pytest


def test_rank_one(orc):
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(7), rng.standard_normal(5)
    A = np.outer(x, y)
    s2 = orc.sigma_max2(A)
    np.testing.assert_allclose(s2, (x @ x) * (y @ y), rtol=1e-12)
    for eta in (1, 2, 10, 1000):
        assert orc.alpha_star(eta, s2, (A ** 2).sum()) == pytest.approx(1.0, rel=1e-12)


def test_orthogonal_equal_rows(orc):
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    A = 3.0 * Q[:5]                      # 5 orthogonal rows of norm 3
    s2 = orc.sigma_max2(A)
    np.testing.assert_allclose(s2, 9.0, rtol=1e-12)
    for eta in (1, 4, 64):
        np.testing.assert_allclose(orc.alpha_star(eta, s2, 45.0), eta / (1 + (eta - 1) / 5),
                                   rtol=1e-12)


def test_diagonal(orc):
    d = np.array([0.5, -4.0, 2.0, 1.0])
    np.testing.assert_allclose(orc.sigma_max2(np.diag(d)), 16.0, rtol=1e-12)
    np.testing.assert_allclose(orc.sigma_max2(np.diag(d)[:, :3]), 16.0, rtol=1e-12)


@pytest.mark.parametrize("eta,s", [(2, 0.3), (16, 0.05), (1024, 0.0015)])
def test_alpha_star_maximises_rate_bound(orc, eta, s):
    L = lambda a: a - a / (2.0 * eta) * (a * (eta - 1) * s + a)
    a = orc.alpha_star(eta, s, 1.0)
    assert L(a) == pytest.approx(eta / (2.0 + 2.0 * (eta - 1) * s), rel=1e-12)
    h = 1e-6 * a
    assert (L(a + h) - L(a - h)) / (2 * h) == pytest.approx(0.0, abs=1e-6)
    assert L(a) >= L(0.9 * a) and L(a) >= L(1.1 * a)
    assert orc.alpha_star(1, s, 1.0) == 1.0
