"""The sweep harness over Sec. 5's experiment settings (experiments.py) on the
GPU: one of its runs against the oracle, and the qualitative claims of Sec. 5
on their own settings with fixed seeds:

* Sec. 5.1: on the overdetermined 100 x 10 system with lambda = 0.01, larger
  eta needs fewer iterations to reach an error of 1e-3 (v2);
* Sec. 5.2 / Theorem th:RSKA: alpha = alpha^*(eta) converges, alpha four
  times larger diverges on the 100 x 10 system with lambda = 6.
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
    from paper_2203_10838_gb300 import experiments
    return torch, oracle, experiments


def test_run_curve_matches_oracle(env):
    torch, orc, ex = env
    p = gaussian_problem(100, 200, 10, seed=5)
    dev = torch.device("cuda")
    A = torch.from_numpy(p.A).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    xh = torch.from_numpy(p.xhat.astype(np.float32)).to(dev)
    its, rr, re = ex.run_curve(A, b, xh, 200, 1.0, 11, 2.0, 3, 300, 50)
    assert list(its) == [0, 50, 100, 150, 200, 250, 300]
    An = p.A[:, :200]
    nu = orc.row_norms(An)
    thr, alias = orc.alias_build(nu)
    for k, r_g, e_g in zip(its[1:], rr[1:], re[1:]):
        tau = orc.sample(thr, alias, seed=3, eta=11, k0=0, K=int(k))
        z = orc.rska_fixed(An, p.b.astype(np.float64), 1.0, 2.0, 11, tau, nu=nu)
        r_o, e_o = orc.metrics(An, p.b.astype(np.float64), z, 1.0, p.xhat)
        assert abs(r_g - r_o) <= 2e-4 * max(1.0, r_o) and abs(e_g - e_o) <= 2e-4 * max(1.0, e_o)


def test_setting_structure_and_variants(env):
    torch, orc, ex = env
    res = ex.run_setting("compare_100x20", trials=2, variants=ex.VARIANTS, K=200)
    assert set(res["runs"]) == set(ex.VARIANTS)
    for label, c in res["runs"].items():
        assert len(c["iterations"]) == len(c["residual_mean"]) == len(c["error_mean"])
        assert c["residual_mean"][-1] < c["residual_mean"][0], label


def test_larger_eta_needs_fewer_iterations(env):
    torch, orc, ex = env
    res = ex.run_setting("eta_100x10_lam0.01", trials=3, etas=(1, 4, 16), K=1500,
                         check_every=10)
    its = [ex.iterations_to(res["runs"][f"v2_eta{e}"], 1e-3) for e in (1, 4, 16)]
    assert all(i is not None for i in its), its
    assert its[0] > its[1] >= its[2], its


def test_alpha_star_converges_and_four_times_it_diverges(env):
    torch, orc, ex = env
    p = gaussian_problem(100, 10, 10, seed=10_000)
    A = p.A[:, :10].astype(np.float64)
    a_star = orc.alpha_star(4, orc.sigma_max2(A), (A ** 2).sum())
    res = ex.run_setting("alpha_eta_100x10", trials=2, etas=(4,), alphas=(a_star, 4 * a_star),
                         K=100, check_every=10)
    good = res["runs"][f"eta4_alpha{a_star:g}"]["residual_mean"]
    bad = res["runs"][f"eta4_alpha{4 * a_star:g}"]["residual_mean"]
    assert good[-1] < 0.5 * good[0]
    assert not (bad[-1] < bad[0])
