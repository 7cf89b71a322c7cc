"""Pins for the oracle's linearized Bregman iteration (the eta -> infinity limit
of eq. rska; Sec. 4 remarks) against facts outside its code:

* one step with step = t/||A||_F^2 equals the exact mean of one RSKA step with
  uniform weights t over all m^eta index tuples (computed by the C oracle);
* with lambda = 0 it converges from z = 0 to the minimum-norm solution A^+ b
  (a library pseudo-inverse);
* on consistent tiny systems it converges to the brute-force solution of the
  regularized basis pursuit problem (eq. RBPP).
"""
import itertools

import numpy as np
import pytest

from test_oracle_rska import brute_force_rbpp


def soft(z, lam):
    return np.sign(z) * np.maximum(np.abs(z) - lam, 0.0)


@pytest.mark.parametrize("eta,t,lam", [(1, 1.0, 0.3), (2, 2.5, 0.0), (3, 1.2, 0.6)])
def test_one_step_is_the_mean_rska_step(orc, eta, t, lam):
    rng = np.random.default_rng(60 + eta)
    A = rng.standard_normal((4, 3)).astype(np.float32)
    b = rng.standard_normal(4)
    z = rng.standard_normal(3)
    A64 = A.astype(np.float64)
    nu = (A64 ** 2).sum(1)
    p = nu / nu.sum()
    mean = np.zeros(3)
    for tup in itertools.product(range(4), repeat=eta):
        mean += np.prod(p[list(tup)]) * orc.rska_fixed(A, b, lam, t, eta, [list(tup)], z0=z)
    z_lb = orc.linearized_bregman(A, b, lam, t / nu.sum(), 1, z0=z)
    np.testing.assert_allclose(z_lb, mean, rtol=1e-12, atol=1e-14)


def test_lambda_zero_gives_minimum_norm_solution(orc):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((5, 9)).astype(np.float32)
    b = rng.standard_normal(5)
    A64 = A.astype(np.float64)
    step = 1.0 / orc.sigma_max2(A64)
    z = orc.linearized_bregman(A, b, 0.0, step, 4000)
    np.testing.assert_allclose(z, np.linalg.pinv(A64) @ b, rtol=0, atol=1e-10)


@pytest.mark.parametrize("seed,lam", [(7, 0.3), (8, 1.0)])
def test_limit_is_brute_force_rbpp_solution(orc, seed, lam):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 5)).astype(np.float32)
    xhat = np.zeros(5)
    xhat[rng.choice(5, 2, replace=False)] = rng.standard_normal(2)
    A64 = A.astype(np.float64)
    b = A64 @ xhat
    z = orc.linearized_bregman(A, b, lam, 1.0 / orc.sigma_max2(A64), 40000)
    np.testing.assert_allclose(soft(z, lam), brute_force_rbpp(A64, b, lam), rtol=0, atol=1e-8)
