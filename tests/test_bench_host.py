"""Host logic of bench.py that decides reported numbers: the plateau rule of
the time-to-plateau workload (with noisy data the RSKA error levels off at a
horizon set by the noise, Sec. 4, so time to a fixed 1e-6 is replaced by time
to 1.05x the plateau).  CPU only."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_flat_tail_is_a_reached_plateau():
    b = _bench()
    errs = list(np.linspace(1.0, 0.1, 50)) + [0.1] * 50
    plat, reached = b.plateau_of(errs)
    assert reached and plat == 0.1


def test_noisy_flat_tail_is_reached():
    b = _bench()
    rng = np.random.default_rng(0)
    errs = list(np.geomspace(1.0, 0.02, 40)) + list(0.02 * (1 + 0.01 * rng.standard_normal(60)))
    plat, reached = b.plateau_of(errs)
    assert reached and abs(plat - 0.02) < 1e-3


def test_still_decreasing_curves_are_not_reached():
    b = _bench()
    assert not b.plateau_of(list(np.exp(-np.arange(100) / 10.0)))[1]
    assert not b.plateau_of(list(np.linspace(1.0, 0.5, 100)))[1]


def test_diverging_curve_is_not_reached():
    b = _bench()
    errs = list(np.geomspace(1.0, 1e6, 99)) + [float("inf")]
    assert not b.plateau_of(errs)[1]


def test_curve_that_never_moved_is_not_reached():
    b = _bench()
    errs = list(1.0 - 1e-4 * np.arange(100))
    assert not b.plateau_of(errs)[1]
