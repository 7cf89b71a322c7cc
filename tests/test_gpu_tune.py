"""GPU checks of the multi-right-hand-side autotuner (rska_mrhs_tune): every
candidate schedule computes the same iteration (each against the FP64 oracle
within 1e-4 with the default high + low operand split), tuning leaves the
iterate and the iteration count unchanged, and a long first solve picks and
caches a schedule by itself."""
import numpy as np
import pytest

from synth import multi_rhs_problem

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10838_gb300 import build
    build.build()
    import oracle
    oracle.build()
    from paper_2203_10838_gb300 import rska
    return torch, oracle, rska


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def apply(h, rska, code):
    d = rska.decode_schedule(code)
    if d["form"] == "persistent":
        h.set_option("form", rska.MRHS_FORM["persistent"])
        h.set_option("gather_sched", d["gather_sched"])
    else:
        h.set_option("form", rska.MRHS_FORM["staged"])
        h.set_option("ksplit", d["ksplit"])
        h.set_option("pdl", d["pdl"])


def problem(torch, m, n, R, s, seed):
    p = multi_rhs_problem(m, n, R, s, seed=seed)
    A = torch.from_numpy(p.A16.view(np.int16)).cuda().view(torch.bfloat16)
    B = torch.from_numpy(p.B).cuda()
    return p, A, B


def oracle_z(orc, p, n, lam, t, eta, seed, K, rows):
    A32 = np.ascontiguousarray(p.A[:, :n])
    nu = orc.row_norms(A32)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    return orc.rska_mrhs(A32, p.B.astype(np.float64), lam, t, eta, tau, nu=nu, rows=rows)


def test_every_candidate_schedule_matches_the_oracle(env):
    torch, orc, rska = env
    m, n, R, eta, lam, t, seed, K = 3000, 2100, 300, 200, 0.5, 8.0, 5, 70
    p, A, B = problem(torch, m, n, R, 30, 17)
    rows = [0, 1, 77, 128, 255, 256, 299]
    Zr = oracle_z(orc, p, n, lam, t, eta, seed, K, rows)
    codes = rska.tune_candidates(n, R, eta, torch.cuda.get_device_properties(0).multi_processor_count)
    assert any(rska.decode_schedule(c)["form"] == "persistent" for c in codes)
    for code in codes:
        with rska.MultiRHS(A, B, lam, eta, t, seed, n=n) as h:
            apply(h, rska, code)
            h.solve(K)
            z = h.get_x()[1].cpu().numpy().astype(np.float64)
        for r, j in enumerate(rows):
            assert rel(z[j], Zr[r]) <= TOL, (rska.decode_schedule(code), j, rel(z[j], Zr[r]))


def test_tuning_keeps_the_state_and_a_long_solve_tunes_itself(env):
    torch, orc, rska = env
    m, n, R, eta, lam, t, seed = 2000, 1000, 200, 128, 0.5, 8.0, 9
    p, A, B = problem(torch, m, n, R, 20, 23)
    rows = list(range(0, 200, 13))
    # explicit tuning in the middle of a run: the run continues as if untuned
    with rska.MultiRHS(A, B, lam, eta, t, seed, n=n) as h:
        h.solve(30)
        code, us = h.tune(16)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert code in rska.tune_candidates(n, R, eta, sms)
        assert us > 0 and h.query("k") == 30 and h.query("tuned_code") == code
        h.solve(40)
        z = h.get_x()[1].cpu().numpy().astype(np.float64)
    Zr = oracle_z(orc, p, n, lam, t, eta, seed, 70, rows)
    for r, j in enumerate(rows):
        assert rel(z[j], Zr[r]) <= TOL, (j, rel(z[j], Zr[r]))
    # a first solve of at least 128 iterations picks a schedule (from the
    # cache entry the explicit tuning left, for this shape and device)
    with rska.MultiRHS(A, B, lam, eta, t, seed, n=n) as h:
        h.solve(130)
        assert h.query("tuned_code") == code
        z = h.get_x()[1].cpu().numpy().astype(np.float64)
    Zr = oracle_z(orc, p, n, lam, t, eta, seed, 130, rows)
    for r, j in enumerate(rows):
        assert rel(z[j], Zr[r]) <= TOL, (j, rel(z[j], Zr[r]))
    # a pinned schedule is never retuned
    with rska.MultiRHS(A, B, lam, eta, t, seed, n=n) as h:
        h.set_option("form", rska.MRHS_FORM["staged"])
        h.solve(130)
        assert h.query("tuned_code") == 0 and h.query("form") == 1
