"""Pin for the oracle's reverse-mode gradient of K unrolled RSKA iterations:
central finite differences of the forward oracle (eq. rska iterated with a
fixed index sequence), in FP64.

For a fixed index sequence and a fixed pattern of active coordinates
(|x^*_j| > lambda) the map (b, lambda) -> x^*_K is affine and t -> x^*_K is a
polynomial, so central differences are exact up to rounding for b and lambda
and O(h^2) for t.  Directions whose +h and -h runs change any mask along the
trajectory are skipped: the loss is not differentiable across those.
"""
import numpy as np
import pytest

from synth import gaussian_problem


def _masks(orc, A, b, lam, t, eta, tau):
    z = np.zeros(A.shape[1])
    out = [np.abs(z) > lam]
    for k in range(tau.shape[0]):
        z = orc.rska_fixed(A, b, lam, t, eta, tau[k:k + 1], z0=z)
        out.append(np.abs(z) > lam)
    return np.array(out)


def _loss(orc, A, b, lam, t, eta, tau, xhat):
    z = orc.rska_fixed(A, b, lam, t, eta, tau)
    x = np.sign(z) * np.maximum(np.abs(z) - lam, 0.0)
    return 0.5 * np.sum((x - xhat) ** 2)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_unrolled_gradient_matches_central_differences(orc, seed):
    prob = gaussian_problem(24, 10, 3, seed=100 + seed, noise=0.01)
    A = prob.A[:, :10]
    b = prob.b64
    lam, t, eta, K = 0.15, 2.0, 4, 30
    nu = orc.row_norms(A)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    loss, gb, glam, gt = orc.unrolled_grad(A, b, lam, t, eta, tau, prob.xhat)
    assert np.isclose(loss, _loss(orc, A, b, lam, t, eta, tau, prob.xhat), rtol=1e-14)
    assert np.any(gb != 0.0)

    def fd(fun, h):
        return (fun(h) - fun(-h)) / (2 * h)

    rng = np.random.default_rng(seed)
    checked = 0
    base_masks = _masks(orc, A, b, lam, t, eta, tau)
    for trial in range(6):
        d = rng.standard_normal(24)
        h = 1e-6
        mp = _masks(orc, A, b + h * d, lam, t, eta, tau)
        mm = _masks(orc, A, b - h * d, lam, t, eta, tau)
        if not (np.array_equal(mp, base_masks) and np.array_equal(mm, base_masks)):
            continue
        got = fd(lambda e: _loss(orc, A, b + e * d, lam, t, eta, tau, prob.xhat), h)
        np.testing.assert_allclose(gb @ d, got, rtol=1e-6, atol=1e-9)
        checked += 1
    assert checked >= 3

    h = 1e-7
    if (np.array_equal(_masks(orc, A, b, lam + h, t, eta, tau), base_masks)
            and np.array_equal(_masks(orc, A, b, lam - h, t, eta, tau), base_masks)):
        got = fd(lambda e: _loss(orc, A, b, lam + e, t, eta, tau, prob.xhat), h)
        np.testing.assert_allclose(glam, got, rtol=1e-6, atol=1e-9)
    h = 1e-6
    if (np.array_equal(_masks(orc, A, b, lam, t + h, eta, tau), base_masks)
            and np.array_equal(_masks(orc, A, b, lam, t - h, eta, tau), base_masks)):
        got = fd(lambda e: _loss(orc, A, b, lam, t + e, eta, tau, prob.xhat), h)
        np.testing.assert_allclose(gt, got, rtol=1e-5, atol=1e-9)


def test_unrolled_gradient_duplicate_rows_add(orc):
    """A row drawn twice in one iteration contributes twice to dL/db."""
    prob = gaussian_problem(6, 4, 2, seed=5)
    A = prob.A[:, :4]
    tau = np.array([[2, 2]] * 5, dtype=np.int32)
    loss, gb, glam, gt = orc.unrolled_grad(A, prob.b64, 0.0, 1.0, 2, tau, prob.xhat + 1.0)
    assert np.count_nonzero(gb) == 1 and gb[2] != 0.0
    h = 1e-6
    e2 = np.zeros(6)
    e2[2] = 1.0
    lp = _loss(orc, A, prob.b64 + h * e2, 0.0, 1.0, 2, tau, prob.xhat + 1.0)
    lm = _loss(orc, A, prob.b64 - h * e2, 0.0, 1.0, 2, tau, prob.xhat + 1.0)
    np.testing.assert_allclose(gb[2], (lp - lm) / (2 * h), rtol=1e-7)
