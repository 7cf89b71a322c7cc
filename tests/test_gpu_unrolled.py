"""GPU parity of the unrolled form and its hand-written adjoint (rska_unrolled_*
behind a torch.autograd.Function) against the FP64 oracle's reverse-mode
gradient of the same K iterations (itself pinned to central finite
differences on the CPU).

Bar: x_K within 1e-4 relative; dL/db, dL/dlambda, dL/dt within 1e-3 relative
(FP32 forward and adjoint against FP64), for L = 1/2 ||x_K - xhat||^2.
"""
import numpy as np
import pytest

from synth import gaussian_problem, pack_batch

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
    from paper_2203_10838_gb300.rska import Unrolled
    return torch, oracle, Unrolled


def rel(a, b):
    return np.linalg.norm(np.atleast_1d(a - b)) / max(np.linalg.norm(np.atleast_1d(b)), 1e-30)


def run(env, shapes, nnz, noise, eta, K, ckpt, lams, ts, seed, check):
    torch, orc, Unrolled = env
    probs = [gaussian_problem(m, n, nnz, seed=700 + i, noise=noise)
             for i, (m, n) in enumerate(shapes)]
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    Ad = torch.from_numpy(A).cuda()
    un = Unrolled(Ad, a_off, m, n, lda, b_off, eta, seed, K, ckpt)
    bd = torch.from_numpy(b).cuda().requires_grad_(True)
    lam = torch.tensor(lams, dtype=torch.float32, device="cuda", requires_grad=True)
    t = torch.tensor(ts, dtype=torch.float32, device="cuda", requires_grad=True)
    x = un(bd, lam, t)
    xo = un.x_off
    xhat = torch.zeros_like(x)
    for p, pr in enumerate(probs):
        xhat[int(xo[p]):int(xo[p]) + pr.n] = torch.from_numpy(pr.xhat.astype(np.float32))
    loss = 0.5 * ((x - xhat) ** 2).sum()
    loss.backward()
    xg = x.detach().cpu().numpy().astype(np.float64)
    gb = bd.grad.cpu().numpy().astype(np.float64)
    glam = lam.grad.cpu().numpy().astype(np.float64)
    gt = t.grad.cpu().numpy().astype(np.float64)
    un.close()
    for p in check:
        pr = probs[p]
        Ap = pr.A[:, :pr.n]
        nu = orc.row_norms(Ap)
        thr, alias = orc.alias_build(nu)
        tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K, problem=p)
        lam_p = float(np.float32(lams[p]))
        t_p = float(np.float32(ts[p]))
        bp = pr.b.astype(np.float64)
        z = orc.rska_fixed(Ap, bp, lam_p, t_p, eta, tau, nu=nu)
        xr = orc.soft_shrink(z, lam_p)
        xhat_p = pr.xhat.astype(np.float32).astype(np.float64)
        loss_o, gb_o, glam_o, gt_o = orc.unrolled_grad(Ap, bp, lam_p, t_p, eta, tau, xhat_p, nu=nu)
        x_p = xg[int(xo[p]):int(xo[p]) + pr.n]
        assert rel(x_p, xr) <= 1e-4, (p, rel(x_p, xr))
        gb_p = gb[int(b_off[p]):int(b_off[p]) + pr.m]
        assert rel(gb_p, gb_o) <= 1e-3, (p, "b", rel(gb_p, gb_o))
        assert rel(glam[p], glam_o) <= 1e-3, (p, "lambda", glam[p], glam_o)
        assert rel(gt[p], gt_o) <= 1e-3, (p, "t", gt[p], gt_o)


def test_unrolled_gradient_small(env):
    shapes = [(256, 128), (300, 61), (200, 200), (129, 40)]
    run(env, shapes, nnz=6, noise=0.01, eta=16, K=40, ckpt=10,
        lams=[0.2, 0.1, 0.3, 0.05], ts=[4.0, 2.0, 3.0, 1.5], seed=5, check=range(4))


def test_unrolled_gradient_full_size_configuration(env):
    """64 problems of 2048 x 1024, 50 nonzeros, 1% noise, K = 200 unrolled
    iterations, eta = 64, checkpoints every 20, lambda = 1, t = 32; 6 problems
    checked against the FP64 oracle gradient."""
    shapes = [(2048, 1024)] * 64
    run(env, shapes, nnz=50, noise=0.01, eta=64, K=200, ckpt=20, lams=[1.0] * 64,
        ts=[32.0] * 64, seed=11, check=[0, 1, 17, 31, 48, 63])


def test_unrolled_column_form_wide_rows(env):
    """n above the row form's 1024 (ragged widths): the column-split kernels."""
    shapes = [(600, 1100), (300, 1501), (900, 1030)]
    run(env, shapes, nnz=10, noise=0.01, eta=32, K=30, ckpt=10,
        lams=[0.5, 0.3, 0.8], ts=[6.0, 3.0, 8.0], seed=21, check=range(3))


def test_unrolled_column_form_large_eta(env):
    """eta = 300, above the row form's 256."""
    shapes = [(1200, 500), (900, 260)]
    run(env, shapes, nnz=10, noise=0.0, eta=300, K=12, ckpt=4,
        lams=[0.5, 0.2], ts=[40.0, 30.0], seed=22, check=range(2))


def test_unrolled_row_form_limits(env):
    """n = 1024 and eta = 256, the row form's limits."""
    shapes = [(2048, 1024), (1500, 1024), (3000, 1000)]
    run(env, shapes, nnz=20, noise=0.01, eta=256, K=24, ckpt=6,
        lams=[1.0, 0.5, 1.5], ts=[60.0, 40.0, 80.0], seed=23, check=range(3))


def test_unrolled_one_cta_per_problem(env):
    """80 problems: more than half the SMs, so every problem runs on one CTA
    instead of a CTA pair."""
    shapes = [(256 + 8 * (i % 7), 128 + 4 * (i % 5)) for i in range(80)]
    run(env, shapes, nnz=6, noise=0.01, eta=16, K=30, ckpt=10, lams=[0.2] * 80,
        ts=[4.0] * 80, seed=24, check=[0, 13, 41, 79])


@pytest.mark.parametrize("K,ckpt", [(12, 1), (12, 12), (1, 1)])
def test_unrolled_checkpoint_extremes_and_degenerate_shapes(env, K, ckpt):
    """Checkpoints after every iteration (the adjoint recomputes nothing), one
    segment spanning all K iterations, and K = 1; the batch holds a single-row
    problem (its row drawn eta times per iteration) and a single-column one
    beside ragged shapes.  With K = 1 two problems end with x_1 = 0 (every mask
    zero) and their exact gradients are zero."""
    shapes = [(40, 24), (1, 5), (6, 1), (33, 17), (64, 64)]
    run(env, shapes, nnz=3, noise=0.01, eta=8, K=K, ckpt=ckpt, lams=[0.05] * 5, ts=[2.0] * 5,
        seed=17, check=range(5))


def test_backward_of_an_older_forward_raises(env):
    """The adjoint differentiates the most recent forward of a context (its
    checkpoints and the b, lambda, t it borrowed).  A backward of an output
    from an earlier forward must raise instead of returning the gradient at
    the later point."""
    torch, orc, Unrolled = env
    probs = [gaussian_problem(64, 32, 3, seed=800 + i, noise=0.01) for i in range(2)]
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    un = Unrolled(torch.from_numpy(A).cuda(), a_off, m, n, lda, b_off, 8, 3, 10, 5)
    b1 = torch.from_numpy(b).cuda().requires_grad_(True)
    b2 = (1.5 * torch.from_numpy(b).cuda()).requires_grad_(True)
    lam = torch.full((2,), 0.1, device="cuda", requires_grad=True)
    t = torch.full((2,), 2.0, device="cuda", requires_grad=True)
    x1 = un(b1, lam, t)
    x2 = un(b2, lam, t)
    with pytest.raises(RuntimeError, match="most recent forward"):
        x1.sum().backward()
    assert b1.grad is None
    x2.sum().backward()
    assert b2.grad is not None and torch.isfinite(b2.grad).all()
    un.close()


def _masks(orc, A, b, lam, t, eta, tau):
    z = np.zeros(A.shape[1])
    out = [np.abs(z) > lam]
    for k in range(tau.shape[0]):
        z = orc.rska_fixed(A, b, lam, t, eta, tau[k:k + 1], z0=z)
        out.append(np.abs(z) > lam)
    return np.array(out)


def test_adjoint_against_central_differences_of_the_gpu_forward(env):
    """dL/db (along a random unit direction per problem), dL/dlambda and
    dL/dt from the hand-written adjoint against FP32 central differences of
    the GPU forward itself with h = 1e-3, at 1e-2 relative.  Directions whose
    +h or -h run changes a mask |z_j| > lambda anywhere along the trajectory
    (decided by the FP64 oracle) are skipped: the loss is not differentiable
    across those.  With the masks fixed, x_K is affine in b and lambda (so the
    central difference of the quadratic loss is exact up to rounding) and a
    polynomial in t."""
    torch, orc, Unrolled = env
    P, mm, nn, s, eta, K, ck, lam0, t0, seed, h = 12, 64, 24, 3, 8, 8, 4, 0.3, 2.0, 41, 1e-3
    probs = [gaussian_problem(mm, nn, s, seed=1300 + i, noise=0.01) for i in range(P)]
    A, a_off, m, n, lda, b, b_off = pack_batch(probs)
    un = Unrolled(torch.from_numpy(A).cuda(), a_off, m, n, lda, b_off, eta, seed, K, ck)
    xo = un.x_off
    xhat = torch.zeros(int(xo[-1]), device="cuda")
    for p, pr in enumerate(probs):
        xhat[int(xo[p]):int(xo[p]) + pr.n] = torch.from_numpy(pr.xhat.astype(np.float32))
    b0 = torch.from_numpy(b).cuda()
    bd = b0.clone().requires_grad_(True)
    lam = torch.full((P,), lam0, device="cuda", requires_grad=True)
    t = torch.full((P,), t0, device="cuda", requires_grad=True)
    x = un(bd, lam, t)
    (0.5 * ((x - xhat) ** 2).sum()).backward()
    gb = bd.grad.cpu().numpy().astype(np.float64)
    glam = lam.grad.cpu().numpy().astype(np.float64)
    gt = t.grad.cpu().numpy().astype(np.float64)

    def losses(bv, lv, tv):
        with torch.no_grad():
            xx = un.forward_raw(bv.contiguous(), lv.contiguous(), tv.contiguous())
        xx = xx.cpu().numpy().astype(np.float64)
        xh = xhat.cpu().numpy().astype(np.float64)
        return np.array([0.5 * np.sum((xx[int(xo[p]):int(xo[p]) + nn]
                                       - xh[int(xo[p]):int(xo[p]) + nn]) ** 2)
                         for p in range(P)])

    rng = np.random.default_rng(5)
    d = np.zeros_like(b)
    for p in range(P):
        v = rng.standard_normal(mm)
        d[int(b_off[p]):int(b_off[p]) + mm] = v / np.linalg.norm(v)
    dd = torch.from_numpy(d.astype(np.float32)).cuda()
    lv = torch.full((P,), lam0, device="cuda")
    tv = torch.full((P,), t0, device="cuda")
    # b +- h d as the GPU holds them (FP32): the loss difference is compared
    # with the gradient times the exact difference of the two FP32 vectors
    b_plus, b_minus = b0 + h * dd, b0 - h * dd
    db = (b_plus.double() - b_minus.double()).cpu().numpy()
    bpl, bmi = b_plus.double().cpu().numpy(), b_minus.double().cpu().numpy()
    dl_b = losses(b_plus, lv, tv) - losses(b_minus, lv, tv)
    # lambda +- h and t +- h as FP32 values: divide by their exact difference
    lv_p, lv_m, tv_p, tv_m = lv + h, lv - h, tv + h, tv - h
    lp, lm = float(lv_p[0].item()), float(lv_m[0].item())
    tp, tm = float(tv_p[0].item()), float(tv_m[0].item())
    fd_l = (losses(b0, lv_p, tv) - losses(b0, lv_m, tv)) / (lp - lm)
    fd_t = (losses(b0, lv, tv_p) - losses(b0, lv, tv_m)) / (tp - tm)
    un.close()

    checked = {"b": [], "lambda": [], "t": []}
    for p, pr in enumerate(probs):
        Ap = pr.A[:, :nn]
        nu = orc.row_norms(Ap)
        thr, alias = orc.alias_build(nu)
        tau = orc.sample(thr, alias, seed=seed, eta=eta, k0=0, K=K, problem=p)
        bp = pr.b.astype(np.float64)
        seg = slice(int(b_off[p]), int(b_off[p]) + mm)
        lf, tf = float(np.float32(lam0)), float(np.float32(t0))
        base = _masks(orc, Ap, bp, lf, tf, eta, tau)
        same = lambda *a: np.array_equal(_masks(orc, Ap, *a, eta, tau), base)  # noqa: E731
        if same(bpl[seg], lf, tf) and same(bmi[seg], lf, tf):
            checked["b"].append((gb[seg] @ db[seg], dl_b[p]))
        if same(bp, lp, tf) and same(bp, lm, tf):
            checked["lambda"].append((glam[p], fd_l[p]))
        if same(bp, lf, tp) and same(bp, lf, tm):
            checked["t"].append((gt[p], fd_t[p]))
    worst = {}
    for kind, pairs in checked.items():
        assert len(pairs) >= 3, (kind, len(pairs))
        scale = max(abs(f) for _, f in pairs)
        errs = [abs(g - f) / max(abs(f), 1e-3 * scale) for g, f in pairs]
        worst[kind] = max(errs)
        assert worst[kind] <= 1e-2, (kind, pairs)
    print(f"adjoint vs FP32 central differences (h = {h}): worst relative error {worst}, "
          f"directions checked {({k: len(v) for k, v in checked.items()})}")
