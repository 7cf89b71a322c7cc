"""Pins for the oracle's weighted step (eq. rska with a general diagonal weight
matrix W = diag(w); Sec. 5, variants v3 and v4) against facts outside the
oracle's code:

* w = 1 and a constant w = c reduce to the uniform-weight step (t and t c) bit
  for bit;
* the exact mean of the step over all m^eta index tuples equals the closed
  forms: v3 (p_i = ||a_i||^2/||A||_F^2) gives (t/||A||_F^2) A^T W (A x - b),
  v4 (p_i proportional to ||a_i||^2/w_i) gives t A^T (A x - b) / sum_j
  ||a_j||^2/w_j, i.e. P W D^-2 = alpha I with alpha = (sum_j ||a_j||^2/w_j)^-1;
* the v4 alias table, built over rho_i = ||a_i||^2 / w_i, reconstructs rho
  normalised.
"""
import itertools

import numpy as np
import pytest


def soft(z, lam):
    return np.sign(z) * np.maximum(np.abs(z) - lam, 0.0)


def _tiny(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal(m)
    w = rng.uniform(0.05, 1.0, m)
    z = rng.standard_normal(n)
    return A, b, w, z


def test_unit_and_constant_weights_reduce_to_uniform_step(orc):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 12)).astype(np.float32)
    b = rng.standard_normal(30)
    tau = rng.integers(0, 30, size=(25, 4))
    z_u = orc.rska_fixed(A, b, 0.3, 1.7, 4, tau)
    z_1 = orc.rska_fixed(A, b, 0.3, 1.7, 4, tau, w=np.ones(30))
    np.testing.assert_array_equal(z_1, z_u)
    c = 0.37
    z_c = orc.rska_fixed(A, b, 0.3, 1.7, 4, tau, w=np.full(30, c))
    z_tc = orc.rska_fixed(A, b, 0.3, 1.7 * c, 4, tau)
    np.testing.assert_array_equal(z_c, z_tc)


def _mean_step(orc, A, b, w, z, lam, t, eta, p):
    """Exact E[z_k - z_{k+1}] over all m^eta tuples drawn i.i.d. from p."""
    m = A.shape[0]
    mean = np.zeros(A.shape[1])
    for tup in itertools.product(range(m), repeat=eta):
        pr = np.prod(p[list(tup)])
        mean += pr * (z - orc.rska_fixed(A, b, lam, t, eta, [list(tup)], z0=z, w=w))
    return mean


@pytest.mark.parametrize("eta,t,lam", [(1, 1.0, 0.3), (2, 1.0, 0.0), (3, 0.8, 0.5)])
def test_v3_mean_step_closed_form(orc, eta, t, lam):
    A, b, w, z = _tiny(4, 3, seed=20 + eta)
    A64 = A.astype(np.float64)
    nu = (A64 ** 2).sum(1)
    p = nu / nu.sum()
    r = A64 @ soft(z, lam) - b
    mean = _mean_step(orc, A, b, w, z, lam, t, eta, p)
    np.testing.assert_allclose(mean, t / nu.sum() * A64.T @ (w * r), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("eta,t,lam", [(1, 1.0, 0.3), (2, 1.0, 0.2), (3, 1.3, 0.0)])
def test_v4_mean_step_closed_form(orc, eta, t, lam):
    A, b, w, z = _tiny(4, 3, seed=40 + eta)
    A64 = A.astype(np.float64)
    nu = (A64 ** 2).sum(1)
    rho = nu / w
    p = rho / rho.sum()
    r = A64 @ soft(z, lam) - b
    mean = _mean_step(orc, A, b, w, z, lam, t, eta, p)
    np.testing.assert_allclose(mean, t / rho.sum() * A64.T @ r, rtol=1e-12, atol=1e-14)


def test_v4_alias_table_reconstructs_coupled_probabilities(orc):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((500, 40)).astype(np.float32)
    w = rng.uniform(0.0, 1.0, 500).astype(np.float32) + np.float32(1e-3)
    nu = orc.row_norms(A)
    rho = nu / w.astype(np.float64)
    thr, alias = orc.alias_build(rho)
    m = rho.shape[0]
    keep = thr.astype(np.float64) / 2.0 ** 32
    prob = np.zeros(m)
    np.add.at(prob, np.arange(m), keep / m)
    np.add.at(prob, alias.astype(np.int64), (1.0 - keep) / m)
    counts = np.bincount(alias, minlength=m) + 1
    np.testing.assert_array_less(np.abs(prob - rho / rho.sum()), counts * 2.0 ** -32 / m + 1e-13)
