"""Pins of the oracle's shared-A multi-right-hand-side form (oracle.rska_mrhs)
against facts that do not come from the oracle itself:

* the matrix form of one step, Z <- Z - (t/eta) A_tau^T D_tau^-2 (A_tau X - B_tau)
  (Sec. 3, A^T M_k (A x - b) applied to all columns), written here with
  numpy matrix products, step by step on a tiny problem;
* one right-hand side reduces to the single-system iteration, and permuting
  the right-hand sides permutes the iterates (the columns do not interact);
* on consistent overdetermined systems every column converges to its own
  planted solution (Ax = b has exactly one solution there, so the RBPP limit
  is xhat_j whatever lambda).
"""
import numpy as np

from synth import multi_rhs_problem


def test_matrix_form_step_by_step(orc):
    rng = np.random.default_rng(4)
    m, n, R, eta, K, lam, t = 12, 7, 3, 4, 6, 0.3, 1.5
    A = rng.standard_normal((m, n)).astype(np.float32)
    B = rng.standard_normal((R, m))
    nu = (A.astype(np.float64) ** 2).sum(axis=1)
    tau = rng.integers(0, m, size=(K, eta)).astype(np.int32)
    Z = np.zeros((n, R))
    A64 = A.astype(np.float64)
    for k in range(K):
        X = np.sign(Z) * np.maximum(np.abs(Z) - lam, 0.0)
        At = A64[tau[k]]                              # eta x n
        Res = At @ X - B[:, tau[k]].T                 # eta x R
        Z = Z - (t / eta) * (At.T @ (Res / nu[tau[k]][:, None]))
    got = orc.rska_mrhs(A, B, lam, t, eta, tau)
    np.testing.assert_allclose(got, Z.T, rtol=1e-12, atol=1e-12)


def test_single_column_and_permutation(orc):
    p = multi_rhs_problem(60, 25, 5, 3, seed=8)
    A = p.A[:, :p.n]
    nu = orc.row_norms(A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=3, eta=6, k0=0, K=40)
    Z = orc.rska_mrhs(A, p.B, 0.2, 1.0, 6, tau)
    for j in range(p.R):
        zj = orc.rska_fixed(A, p.B[j].astype(np.float64), 0.2, 1.0, 6, tau)
        np.testing.assert_array_equal(Z[j], zj)
    perm = np.array([3, 0, 4, 2, 1])
    Zp = orc.rska_mrhs(A, p.B[perm], 0.2, 1.0, 6, tau)
    np.testing.assert_array_equal(Zp, Z[perm])


def test_consistent_columns_reach_their_planted_solutions(orc):
    p = multi_rhs_problem(240, 40, 4, 4, seed=9)
    A = p.A[:, :p.n]
    nu = orc.row_norms(A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=1, eta=8, k0=0, K=3000)
    Z = orc.rska_mrhs(A, p.B64, 0.5, 1.0, 8, tau)
    X = orc.soft_shrink(Z, 0.5)
    for j in range(p.R):
        err = np.linalg.norm(X[j] - p.Xhat[j]) / np.linalg.norm(p.Xhat[j])
        assert err < 1e-8, (j, err)
