"""Host logic of the sweep harness over Sec. 5's settings (experiments.py),
CPU only: how each variant maps to (lambda, eta, t, weights) and how the
first iteration reaching a tolerance is read off a mean curve."""
import math

import pytest


@pytest.fixture(scope="module")
def ex():
    from paper_2203_10838_gb300 import experiments
    return experiments


def test_variant_parameters(ex, orc):
    lam, eta, s2, f2 = 0.7, 16, 3.0, 40.0
    assert ex._variant_params("rk", lam, eta, s2, f2) == (0.0, 1, 1.0, None)
    assert ex._variant_params("rsk", lam, eta, s2, f2) == (lam, 1, 1.0, None)
    assert ex._variant_params("v1", lam, eta, s2, f2) == (lam, eta, 1.0, None)
    l2, e2, t2, w2 = ex._variant_params("v2", lam, eta, s2, f2)
    assert (l2, e2, w2) == (lam, eta, None)
    assert t2 == pytest.approx(orc.alpha_star(eta, s2, f2), rel=1e-15)   # Corollary 1
    assert ex._variant_params("v3", lam, eta, s2, f2) == (lam, eta, 1.0, "v3")
    assert ex._variant_params("v4", lam, eta, s2, f2) == (lam, eta, 1.0, "v4")
    with pytest.raises(ValueError):
        ex._variant_params("v5", lam, eta, s2, f2)


def test_iterations_to(ex):
    curve = {"iterations": [0, 10, 20, 30], "error_mean": [1.0, 0.1, float("nan"), 1e-4]}
    assert ex.iterations_to(curve, 0.5) == 10
    assert ex.iterations_to(curve, 1e-3) == 30       # the NaN check is skipped
    assert ex.iterations_to(curve, 1e-6) is None
    assert ex.iterations_to({"iterations": [0, 5], "residual_mean": [2.0, 0.5]}, 1.0,
                            key="residual_mean") == 5


def test_settings_follow_the_captions(ex):
    for name, cfg in ex.SETTINGS.items():
        assert cfg["m"] > 0 and cfg["n"] > 0 and 0 < cfg["s"] <= cfg["n"], name
        assert cfg["noise"] in (0.0, 0.1), name
        assert cfg["lam"] is None or cfg["lam"] > 0, name
        assert cfg["eta"] is None or 1 <= cfg["eta"] <= cfg["m"], name
        assert cfg["K"] > 0 and not math.isnan(cfg["K"]), name
