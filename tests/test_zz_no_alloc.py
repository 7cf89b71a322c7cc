"""GPU test of rska_solve_noalloc, the entry point for callers that cannot
allocate device memory while they run (an external memory budget or custom
allocator that forbids cudaMalloc, or code that must not synchronize the device
as cudaMalloc/cudaFree may).  It keeps its working memory in a fixed device
array inside the library.

The test calls it through the C ABI twice in a row, on two different problems
(the second takes the column-split kernel, n > 10240), and checks each result
against the regular entry points (rska_setup + rska_solve + rska_get_x) on the
same inputs, within the parity tolerance of the other GPU tests.  The second
call also shows that a call does not inherit state from the previous one.
This file is collected last so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from synth import gaussian_problem

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_10838_gb300 import build
    build.build()
    from paper_2203_10838_gb300._lib import lib
    from paper_2203_10838_gb300.rska import Solver
    return torch, lib(), Solver


def _regular(torch, Solver, A, b, n, lam, eta, t, seed, K):
    with Solver(A, b, lam, eta, t, seed, n=n) as sol:
        sol.solve(K)
        x, z = sol.get_x()
    return x.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64)


def _noalloc(torch, L, A, b, n, lam, eta, t, seed, K):
    m, lda = A.shape
    x = torch.empty(n, dtype=torch.float32, device=A.device)
    z = torch.empty(n, dtype=torch.float32, device=A.device)
    stream = torch.cuda.current_stream()
    rc = L.rska_solve_noalloc(ctypes.c_void_p(A.data_ptr()), m, n, lda,
                              ctypes.c_void_p(b.data_ptr()), lam, eta, t, seed, K,
                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                              ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.rska_strerror(rc)
    return x.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_noalloc_matches_regular_entry_points_on_two_calls(env):
    torch, L, Solver = env
    cases = [
        # m, n, nnz, eta, lambda, t, seed, K, noise
        (3000, 2000, 40, 64, 1.0, 32.0, 11, 300, 0.0),
        (1200, 12000, 60, 128, 0.05, 60.0, 12, 300, 0.01),
    ]
    for m, n, s, eta, lam, t, seed, K, noise in cases:
        prob = gaussian_problem(m, n, s, seed=500 + seed, noise=noise)
        A = torch.from_numpy(prob.A).cuda()
        b = torch.from_numpy(prob.b).cuda()
        x_na, z_na = _noalloc(torch, L, A, b, n, lam, eta, t, seed, K)
        x_rg, z_rg = _regular(torch, Solver, A, b, n, lam, eta, t, seed, K)
        assert np.linalg.norm(x_rg) > 0
        assert rel(x_na, x_rg) <= REL_TOL, (m, n, rel(x_na, x_rg))
        assert rel(z_na, z_rg) <= REL_TOL, (m, n, rel(z_na, z_rg))


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, L, Solver = env
    A = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    b = torch.zeros(4, dtype=torch.float32, device="cuda")
    x = torch.empty(8, dtype=torch.float32, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # m above the limit: rejected on the host before any device work
    assert L.rska_solve_noalloc(p(A), 70000, 8, 8, p(b), 1.0, 4, 1.0, 0, 1, p(x), None,
                                None) == 7
    assert L.rska_solve_noalloc(p(A), 4, 8, 8, p(b), 1.0, 2048, 1.0, 0, 1, p(x), None,
                                None) == 7


def test_noalloc_runs_several_launches_like_the_regular_path(env):
    """eta = 1024 gives 64 iterations per launch of the allocation-free path
    (its pre-sampled index buffer holds 65536 draws), so K = 200 takes four
    launches; from the second on, each continues the index sequence from the
    iteration counter the previous launch left on the device.  The result
    must still match the regular entry points."""
    torch, L, Solver = env
    m, n, s, eta, lam, t, seed, K = 6000, 3000, 50, 1024, 1.0, 400.0, 13, 200
    prob = gaussian_problem(m, n, s, seed=513, noise=0.01)
    A = torch.from_numpy(prob.A).cuda()
    b = torch.from_numpy(prob.b).cuda()
    x_na, z_na = _noalloc(torch, L, A, b, n, lam, eta, t, seed, K)
    x_rg, z_rg = _regular(torch, Solver, A, b, n, lam, eta, t, seed, K)
    assert np.linalg.norm(x_rg) > 0
    assert rel(x_na, x_rg) <= REL_TOL, rel(x_na, x_rg)
    assert rel(z_na, z_rg) <= REL_TOL, rel(z_na, z_rg)
