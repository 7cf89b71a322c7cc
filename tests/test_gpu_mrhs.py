"""GPU parity of the shared-A multi-right-hand-side tensor-core path
(rska_mrhs_*) against the FP64 oracle (oracle.rska_mrhs: eq. (rska) per
right-hand side with the one shared index sequence, on the BF16-valued A
widened to FP64).

Bar: row norms, alias table and tau bit-exact; after K iterations every
checked right-hand side within 5e-3 relative of the oracle's x_K (the BF16-A
tolerance); with the default hi+lo split of the inexact operands also within
1e-4.  The first product's partial tiles are added with atomics, so two runs
agree to rounding, not bit for bit.
"""
import numpy as np
import pytest

from synth import multi_rhs_problem

pytestmark = pytest.mark.gpu

SPEC_TOL = 5e-3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10838_gb300 import build
    build.build()
    import oracle
    oracle.build()
    from paper_2203_10838_gb300.rska import MultiRHS
    return torch, oracle, MultiRHS


def to_dev(torch, p):
    A = torch.from_numpy(p.A16.view(np.int16)).cuda().view(torch.bfloat16)
    B = torch.from_numpy(p.B).cuda()
    return A, B


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


FORMS = ["staged", "persistent"]


def run_case(env, m, n, R, s, eta, lam, t, K, seed, check_rows, tol, terms=2, pseed=21,
             form="auto", terms_update=0):
    torch, orc, MultiRHS = env
    from paper_2203_10838_gb300.rska import MRHS_FORM
    p = multi_rhs_problem(m, n, R, s, seed=pseed)
    A, B = to_dev(torch, p)
    with MultiRHS(A, B, lam, eta, t, seed, n=n) as h:
        h.set_option("form", MRHS_FORM[form])
        if form != "auto":
            assert h.query("form") == MRHS_FORM[form]
        h.set_option("terms", terms)
        h.set_option("terms_update", terms_update)
        nu_g, thr_g, al_g = [v.cpu().numpy() for v in h.get_tables()]
        tau_g = h.get_indices(0, K).cpu().numpy()
        h.solve(K)
        x, z = [v.cpu().numpy().astype(np.float64) for v in h.get_x()]
    A32 = np.ascontiguousarray(p.A[:, :n])
    nu = orc.row_norms(A32)
    thr, alias = orc.alias_build(nu)
    tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K)
    np.testing.assert_array_equal(nu_g, nu)
    np.testing.assert_array_equal(thr_g.view(np.uint32), thr)
    np.testing.assert_array_equal(al_g, alias)
    np.testing.assert_array_equal(tau_g, tau)
    Bf = p.B.astype(np.float64)
    Zr = orc.rska_mrhs(A32, Bf, lam, t, eta, tau, nu=nu, rows=check_rows)
    worst = 0.0
    for r, j in enumerate(check_rows):
        xr = orc.soft_shrink(Zr[r], lam)
        e = rel(x[j], xr) if np.linalg.norm(xr) > 0 else np.abs(x[j]).max()
        worst = max(worst, e)
        assert e <= tol, (j, e)
        assert rel(z[j], Zr[r]) <= tol, (j, rel(z[j], Zr[r]))
    return worst, x


@pytest.mark.parametrize("K", [1, 2, 5])
def test_mrhs_persistent_first_iterations(env, K):
    """The first iterations of the persistent form one by one (lambda = 0, so
    x = z and both products see nonzero operands from the second iteration
    on): 128 right-hand sides on two column slices, eta = 64."""
    run_case(env, 600, 512, 128, 8, eta=64, lam=0.0, t=2.0, K=K, seed=9,
             check_rows=range(0, 128, 5), tol=1e-4, form="persistent")


@pytest.mark.parametrize("form", FORMS)
def test_mrhs_small_ragged(env, form):
    # n = 300 (padded to 512), eta = 100 (padded to 128 / 128), R = 40 (padded to 256)
    run_case(env, 700, 300, 40, 10, eta=100, lam=0.3, t=1.0, K=30, seed=7,
             check_rows=range(40), tol=1e-4, form=form)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("m,n,R,eta", [(5, 3, 1, 1), (1, 7, 3, 3)])
def test_mrhs_degenerate_shapes(env, m, n, R, eta, form):
    """One right-hand side with eta = 1 on a 5 x 3 system (every operand a
    sliver of its padded tile), and a single row drawn eta times per iteration
    for three right-hand sides."""
    run_case(env, m, n, R, 1, eta=eta, lam=0.001, t=1.0, K=40, seed=3,
             check_rows=range(R), tol=1e-4, form=form)


@pytest.mark.parametrize("form", FORMS)
def test_mrhs_single_term_within_spec(env, form):
    run_case(env, 700, 300, 40, 10, eta=100, lam=0.3, t=1.0, K=30, seed=7,
             check_rows=range(40), tol=SPEC_TOL, terms=1, form=form)


def test_mrhs_single_term_update_within_spec(env):
    """X as high + low parts, the scaled residual as one BF16 term."""
    run_case(env, 700, 300, 40, 10, eta=100, lam=0.3, t=1.0, K=30, seed=7,
             check_rows=range(40), tol=SPEC_TOL, terms=2, terms_update=1, form="persistent")


@pytest.mark.parametrize("form", FORMS)
def test_mrhs_several_tiles(env, form):
    # 9 column tiles of the update product, 2 right-hand-side tiles, eta = 2 x 128
    run_case(env, 3000, 2100, 300, 50, eta=256, lam=0.5, t=8.0, K=20, seed=5,
             check_rows=[0, 1, 77, 128, 255, 256, 299], tol=1e-4, form=form)


@pytest.mark.parametrize("form", FORMS)
def test_mrhs_full_size_configuration(env, form):
    """A 16384 x 8192 N(0, 1/n) in BF16, 512 right-hand sides with 400
    nonzeros each, lambda = 1, eta = 256, t = 128; 50 iterations, 16
    right-hand sides checked against the FP64 oracle."""
    run_case(env, 16384, 8192, 512, 400, eta=256, lam=1.0, t=128.0, K=50, seed=0,
             check_rows=list(range(0, 512, 32)), tol=1e-4, pseed=1, form=form)


def test_mrhs_persistent_launch_boundaries_and_form_switches(env):
    """One persistent launch runs at most 512 iterations: 600 iterations in
    one call (two launches), in uneven calls, and alternating between the
    staged and the persistent form (the staged form's X is rebuilt from Z
    after persistent launches) all give the same iterate."""
    torch, orc, MultiRHS = env
    from paper_2203_10838_gb300.rska import MRHS_FORM
    p = multi_rhs_problem(900, 500, 64, 12, seed=3)
    A, B = to_dev(torch, p)
    outs = []
    plans = [[("persistent", 600)], [("persistent", 100), ("persistent", 500)],
             [("staged", 130), ("persistent", 300), ("staged", 70), ("persistent", 100)],
             [("staged", 600)]]
    for plan in plans:
        with MultiRHS(A, B, 0.3, 64, 2.0, 11, n=500) as h:
            for form, k in plan:
                h.set_option("form", MRHS_FORM[form])
                h.solve(k)
            assert h.query("k") == 600
            outs.append(h.get_x()[1].cpu().numpy().astype(np.float64))
    for o in outs[1:]:
        assert rel(o, outs[0]) <= 1e-4


def test_mrhs_resume_and_graph_agree(env):
    torch, orc, MultiRHS = env
    p = multi_rhs_problem(900, 500, 64, 12, seed=3)
    A, B = to_dev(torch, p)
    outs = []
    from paper_2203_10838_gb300.rska import MRHS_FORM
    for graph, chunks in [(1, [70]), (0, [70]), (1, [30, 40])]:
        with MultiRHS(A, B, 0.3, 64, 2.0, 11, n=500) as h:
            h.set_option("form", MRHS_FORM["staged"])
            h.set_option("graph", graph)
            for c in chunks:
                h.solve(c)
            assert h.query("k") == 70
            outs.append(h.get_x()[1].cpu().numpy().astype(np.float64))
    for o in outs[1:]:
        assert rel(o, outs[0]) <= 1e-5


def test_mrhs_rejects_bad_data(env):
    torch, orc, MultiRHS = env
    from paper_2203_10838_gb300._lib import RSKAError
    p = multi_rhs_problem(50, 16, 3, 2, seed=2)
    p.A16[7] = 0
    A, B = to_dev(torch, p)
    with pytest.raises(RSKAError) as e:
        MultiRHS(A, B, 0.1, 8, 1.0, 0, n=16)
    assert e.value.code == 2
    p = multi_rhs_problem(50, 16, 3, 2, seed=2)
    p.B[1, 3] = np.inf
    A, B = to_dev(torch, p)
    with pytest.raises(RSKAError) as e:
        MultiRHS(A, B, 0.1, 8, 1.0, 0, n=16)
    assert e.value.code == 3
