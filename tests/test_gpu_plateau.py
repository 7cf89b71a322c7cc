"""The time-to-plateau measure of the benchmark (with 1% noise the RSKA error
levels off at a horizon set by the noise, Sec. 4, instead of reaching 1e-6)
on the GPU against the oracle's FP64 error curve for the same index sequence.

Bar: the FP64 relative errors of the two curves agree within 2% at every
check (the plateau sits near 1e-3, where FP32 rounding of x is a visible share
of the error), both curves reach a plateau by the benchmark's rule, the two
plateaus agree within 2% and the first checks at or below 1.05x the plateau
lie within 5 checks of each other.
"""
import importlib.util
import os

import numpy as np
import pytest

from synth import gaussian_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10838_gb300 import build
    build.build()
    import oracle
    oracle.build()
    from paper_2203_10838_gb300.rska import Solver
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return torch, oracle, Solver, bench


def test_plateau_time_matches_oracle(env):
    torch, orc, Solver, bench = env
    m, n, s, lam, eta, seed, checks = 2000, 1000, 20, 2.0, 256, 7, 100
    p = gaussian_problem(m, n, s, seed=4242, noise=0.01)
    An = np.ascontiguousarray(p.A[:, :n])
    b64 = p.b.astype(np.float64)
    nu = orc.row_norms(An)
    thr, alias = orc.alias_build(nu)
    t = orc.alpha_star(eta, orc.sigma_max2(An), nu.sum())
    C = -(-m // eta)

    z = None
    e_orc = []
    for j in range(checks):
        z = orc.rska(An, b64, lam, eta, t, seed, C, k0=j * C, z0=z, tables=(nu, thr, alias))
        e_orc.append(orc.metrics(An, b64, z, lam, p.xhat)[1])

    dev = torch.device("cuda")
    xh = torch.from_numpy(p.xhat.astype(np.float32)).to(dev)
    e_gpu = []
    with Solver(torch.from_numpy(p.A).to(dev), torch.from_numpy(p.b).to(dev), lam, eta, t, seed,
                n=n) as sol:
        for _ in range(checks):
            sol.solve(C)
            e_gpu.append(sol.metrics(xh)[1])

    e_orc, e_gpu = np.array(e_orc), np.array(e_gpu)
    assert np.max(np.abs(e_gpu - e_orc) / e_orc) <= 0.02, np.max(np.abs(e_gpu - e_orc) / e_orc)
    plat_o, ok_o = bench.plateau_of(e_orc)
    plat_g, ok_g = bench.plateau_of(e_gpu)
    assert ok_o and ok_g, (plat_o, plat_g)
    assert abs(plat_g - plat_o) <= 0.02 * plat_o, (plat_g, plat_o)
    first_o = int(np.argmax(e_orc <= 1.05 * plat_o))
    first_g = int(np.argmax(e_gpu <= 1.05 * plat_g))
    assert abs(first_g - first_o) <= 5, (first_g, first_o)
