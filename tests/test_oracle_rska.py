"""Pins for the oracle's RSKA iteration (eq. rska, Algorithm 1) against what the
paper and the mathematics fix, independently of the oracle's own code:

* a hand-worked two-step example (tests/golden/rska_2x2_two_steps.json);
* exact first and second moments of the step over all m^eta index tuples
  (Lemma 1 / Lemma 2) and the expected Bregman decrease (Lemma lm:bd);
* eta = 1 is RSK (eq. rsk), lambda = 0 converges to the minimum-norm solution
  A^+ b (a library pseudo-inverse), x^*_k stays in range(A^T) (Sec. 3, the
  matrix form x^*_{k+1} = x^*_k - A^T M_k (A x_k - b));
* the limit equals a brute-force solution of the regularized basis pursuit
  problem (eq. RBPP), enumerated over sign patterns.
"""
import itertools
import json
import os

import numpy as np
import pytest

from synth import gaussian_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def soft(z, lam):
    return np.sign(z) * np.maximum(np.abs(z) - lam, 0.0)


def test_golden_two_steps(orc):
    g = json.load(open(os.path.join(GOLDEN, "rska_2x2_two_steps.json")))
    A = np.array(g["A"], np.float32)
    b = np.array(g["b"])
    z1 = orc.rska_fixed(A, b, g["lambda"], g["t"], g["eta"], [g["tau"][0]], z0=g["z0"])
    np.testing.assert_allclose(z1, g["z1"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(soft(z1, g["lambda"]), g["x1"], rtol=0, atol=1e-15)
    z2 = orc.rska_fixed(A, b, g["lambda"], g["t"], g["eta"], g["tau"], z0=g["z0"])
    np.testing.assert_allclose(z2, g["z2"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(soft(z2, g["lambda"]), g["x2"], rtol=0, atol=1e-15)


def _tiny(m, n, seed, consistent=True, s=2):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)).astype(np.float32)
    xhat = np.zeros(n)
    xhat[rng.choice(n, s, replace=False)] = rng.standard_normal(s)
    b = A.astype(np.float64) @ xhat
    if not consistent:
        b = b + 0.3 * rng.standard_normal(m)
    return A, b, xhat


def _enumerate_step(orc, A, b, lam, t, eta, z):
    """All m^eta index tuples with their probabilities p_i = ||a_i||^2/||A||_F^2
    and the resulting z_{k+1}."""
    A64 = A.astype(np.float64)
    m = A.shape[0]
    nu = (A64 ** 2).sum(1)
    p = nu / nu.sum()
    out = []
    for tup in itertools.product(range(m), repeat=eta):
        w = np.prod(p[list(tup)])
        z1 = orc.rska_fixed(A, b, lam, t, eta, [list(tup)], z0=z)
        out.append((w, z1))
    return out


@pytest.mark.parametrize("eta,t,lam", [(1, 1.0, 0.4), (2, 1.7, 0.0), (3, 2.2, 0.4)])
def test_step_moments_match_lemma_1(orc, eta, t, lam):
    """E[delta] = (t/||A||_F^2) A^T (A x - b) and
    E||delta||^2 = r^T [(1/eta) t^2/||A||_F^2 I + t^2 (1-1/eta) A A^T/||A||_F^4] r
    for w_i = t and p_i = ||a_i||^2/||A||_F^2 (Lemma 1 with Assumption 1)."""
    A, b, _ = _tiny(4, 3, seed=eta, consistent=False)
    rng = np.random.default_rng(10 + eta)
    z = rng.standard_normal(3)
    x = soft(z, lam)
    A64 = A.astype(np.float64)
    F2 = (A64 ** 2).sum()
    r = A64 @ x - b
    mean = np.zeros(3)
    second = 0.0
    for w, z1 in _enumerate_step(orc, A, b, lam, t, eta, z):
        d = z - z1
        mean += w * d
        second += w * d @ d
    np.testing.assert_allclose(mean, t / F2 * A64.T @ r, rtol=1e-12, atol=1e-14)
    Mexp = t * t / (eta * F2) * np.eye(4) + t * t * (1 - 1 / eta) * (A64 @ A64.T) / F2 ** 2
    np.testing.assert_allclose(second, r @ Mexp @ r, rtol=1e-12)


def _bregman(z, y, lam):
    """D_f^{z}(x, y) = f(y) - f(x) - <z, y - x>, x = S_lam(z), f = lam||.||_1 + 1/2||.||^2
    (Definition def:D; z is a subgradient of f at x)."""
    x = soft(z, lam)
    f = lambda v: lam * np.abs(v).sum() + 0.5 * v @ v
    return f(y) - f(x) - z @ (y - x)


@pytest.mark.parametrize("eta,t", [(2, 1.0), (3, 1.8)])
def test_expected_bregman_decrease_lemma_bd(orc, eta, t):
    """E[D(x_{k+1}, xhat)] <= D(x_k, xhat) - (t/||A||_F^2)(1 - s_max(T)) ||A x_k - b||^2
    with T = (1/2eta) W + (t/2)(1 - 1/eta) A A^T/||A||_F^2, W = t I (Lemma lm:bd)."""
    lam = 0.3
    A, b, xhat = _tiny(5, 3, seed=20 + eta, consistent=True)
    A64 = A.astype(np.float64)
    F2 = (A64 ** 2).sum()
    T = np.eye(5) * t / (2 * eta) + t / 2 * (1 - 1 / eta) * (A64 @ A64.T) / F2
    smax = np.linalg.eigvalsh(T).max()
    rng = np.random.default_rng(eta)
    for trial in range(3):
        z = A64.T @ rng.standard_normal(5)          # a reachable dual iterate
        x = soft(z, lam)
        lhs = sum(w * _bregman(z1, xhat, lam) for w, z1 in _enumerate_step(orc, A, b, lam, t, eta, z))
        res = A64 @ x - b
        rhs = _bregman(z, xhat, lam) - t / F2 * (1 - smax) * (res @ res)
        assert lhs <= rhs + 1e-12 * max(1.0, abs(rhs)), (lhs, rhs)


def test_sigma_max_T_closed_form():
    """Lemma lm:svt for W = alpha I: s_max(T) = (1/2eta)(alpha + alpha (eta-1) s_max(A)^2/||A||_F^2)."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 4))
    F2 = (A ** 2).sum()
    s2 = np.linalg.svd(A, compute_uv=False)[0] ** 2
    for eta, alpha in [(1, 1.0), (4, 2.5), (9, 5.0)]:
        T = np.eye(6) * alpha / (2 * eta) + alpha / 2 * (1 - 1 / eta) * (A @ A.T) / F2
        np.testing.assert_allclose(np.linalg.eigvalsh(T).max(),
                                   (alpha + alpha * (eta - 1) * s2 / F2) / (2 * eta), rtol=1e-12)


def test_eta_one_is_rsk(orc):
    """eta = 1, w = 1 recovers standard RSK, eq. (rsk) (Sec. 1.1)."""
    A, b, _ = _tiny(6, 4, seed=3, consistent=False)
    A64 = A.astype(np.float64)
    lam = 0.25
    rng = np.random.default_rng(4)
    tau = rng.integers(0, 6, size=(40, 1))
    z = orc.rska_fixed(A, b, lam, 1.0, 1, tau)
    zs = np.zeros(4)
    for (i,) in tau:
        xs = soft(zs, lam)
        zs = zs - (A64[i] @ xs - b[i]) / (A64[i] @ A64[i]) * A64[i]
    np.testing.assert_allclose(z, zs, rtol=1e-13, atol=1e-14)


def test_lambda_zero_converges_to_minimum_norm_solution(orc):
    """lambda = 0: x = x^*, randomized (averaged) Kaczmarz from 0 converges to
    A^+ b on a consistent underdetermined system (Sec. 1.1, eq. rk)."""
    A, b, _ = _tiny(4, 7, seed=5, s=3)
    z = orc.rska(A, b, 0.0, eta=3, t=1.0, seed=1, K=20000)
    np.testing.assert_allclose(z, np.linalg.pinv(A.astype(np.float64)) @ b, rtol=0, atol=1e-10)


def test_dual_iterate_stays_in_row_space(orc):
    """x^*_k = -sum A^T M_j (A x_j - b) lies in range(A^T) (matrix form, Sec. 3)."""
    A, b, _ = _tiny(4, 9, seed=6, consistent=False)
    z = orc.rska(A, b, 0.5, eta=2, t=1.3, seed=3, K=300)
    A64 = A.astype(np.float64)
    P = np.eye(9) - np.linalg.pinv(A64) @ A64
    assert np.linalg.norm(P @ z) <= 1e-12 * np.linalg.norm(z)
    assert np.linalg.norm(z) > 0


def brute_force_rbpp(A, b, lam):
    """min lam||x||_1 + 1/2||x||^2 s.t. Ax = b (eq. RBPP) by enumerating sign
    patterns: for each pattern solve the equality-constrained quadratic on its
    support, keep feasible sign-consistent candidates, return the best."""
    m, n = A.shape
    best, best_x = np.inf, None
    for sig in itertools.product((-1, 0, 1), repeat=n):
        sig = np.array(sig, dtype=np.float64)
        S = np.flatnonzero(sig)
        if S.size == 0:
            if np.linalg.norm(b) < 1e-12:
                return np.zeros(n)
            continue
        AS = A[:, S]
        k = S.size
        K = np.zeros((k + m, k + m))
        K[:k, :k] = np.eye(k)
        K[:k, k:] = AS.T
        K[k:, :k] = AS
        rhs = np.concatenate([-lam * sig[S], b])
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
        xS = sol[:k]
        if np.linalg.norm(AS @ xS - b) > 1e-9 * max(1.0, np.linalg.norm(b)):
            continue
        if np.any(np.sign(xS) != sig[S]):
            continue
        x = np.zeros(n)
        x[S] = xS
        obj = lam * np.abs(x).sum() + 0.5 * x @ x
        if obj < best:
            best, best_x = obj, x
    return best_x


@pytest.mark.parametrize("seed,lam", [(7, 0.3), (8, 1.0), (9, 0.05)])
def test_limit_is_brute_force_rbpp_solution(orc, seed, lam):
    """Consistent systems: the iterates converge to the unique RBPP solution
    (Theorem th:RSKA)."""
    A, b, _ = _tiny(3, 5, seed=seed, s=2)
    A64 = A.astype(np.float64)
    xbf = brute_force_rbpp(A64, b, lam)
    z = orc.rska(A, b, lam, eta=2, t=1.0, seed=seed, K=60000)
    np.testing.assert_allclose(soft(z, lam), xbf, rtol=0, atol=1e-8)


def test_overdetermined_consistent_recovers_planted_solution(orc):
    prob = gaussian_problem(40, 12, 3, seed=12)
    A = prob.A[:, :12]
    b = prob.b64
    z = orc.rska(A, b, 1.0, eta=4, t=3.0, seed=2, K=6000)
    np.testing.assert_allclose(soft(z, 1.0), prob.xhat, rtol=0, atol=1e-9)
    rr, re = orc.metrics(A, b, z, 1.0, prob.xhat)
    assert rr < 1e-9 and re < 1e-9


def test_sampled_equals_fixed_with_drawn_indices(orc):
    prob = gaussian_problem(30, 17, 4, seed=13)
    A = prob.A[:, :17]
    nu = orc.row_norms(A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=77, eta=5, k0=3, K=25)
    z_fixed = orc.rska_fixed(A, prob.b64, 0.7, 2.0, 5, tau)
    z_samp = orc.rska(A, prob.b64, 0.7, eta=5, t=2.0, seed=77, K=25, k0=3)
    np.testing.assert_array_equal(z_fixed, z_samp)
    # resuming from a checkpoint continues the same index sequence
    z_a = orc.rska(A, prob.b64, 0.7, eta=5, t=2.0, seed=77, K=10, k0=3)
    z_b = orc.rska(A, prob.b64, 0.7, eta=5, t=2.0, seed=77, K=15, k0=13, z0=z_a)
    np.testing.assert_array_equal(z_b, z_samp)


def test_padding_columns_are_ignored(orc):
    prob = gaussian_problem(20, 9, 2, seed=14, lda=16)
    A = prob.A.copy()
    A[:, 9:] = 123.0   # garbage in the padding must not matter when n is passed
    import ctypes
    lib = orc._load()
    nu = np.zeros(20)
    lib.orc_row_norms(orc._ptr(A), 20, 9, 16, orc._ptr(nu))
    np.testing.assert_allclose(nu, (A[:, :9].astype(np.float64) ** 2).sum(1), rtol=1e-15)


def test_metrics_closed_form(orc):
    A = np.array([[1.0, 0.0], [0.0, 2.0]], np.float32)
    b = np.array([3.0, 4.0])
    z = np.array([2.5, -1.5])       # x = S_0.5(z) = (2, -1)
    rr, re = orc.metrics(A, b, z, 0.5, xhat=np.array([2.0, 2.0]))
    # A x - b = (-1, -6); ||.|| = sqrt(37); ||b|| = 5; x - xhat = (0, -3)
    np.testing.assert_allclose(rr, np.sqrt(37) / 5, rtol=1e-15)
    np.testing.assert_allclose(re, 3 / np.sqrt(8), rtol=1e-15)
