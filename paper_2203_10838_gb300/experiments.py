"""Sweeps over the settings of the paper's experiments (Sec. 5), run on the GPU
through the public API.

Every setting is a seeded synthetic system with the shapes and parameters of
one of Sec. 5's figures (A i.i.d. N(0, 1), an s-sparse xhat with N(0, 1)
values, b = A xhat plus optional relative noise), optionally scaled up by a
factor applied to m, n and s.  Each run records the relative residual
||A x - b|| / ||b|| and the error ||x - xhat|| / ||xhat|| (FP64 on the device)
every ``check_every`` iterations; trials differ in their data and Philox seeds
and are summarised by their mean and standard deviation, as the figures do.

Variants (Sec. 5): RK (eta = 1, lambda = 0), RSK (eta = 1), RSKA v1 (t = 1),
v2 (t = alpha^*(eta) from a power-iteration estimate of sigma_max(A)^2,
Corollary 1), v3 and v4 (row weights w_i ~ U[0, 1], probabilities by ||a_i||^2
resp. ||a_i||^2 / w_i).

    python -m paper_2203_10838_gb300.experiments --setting eta_200x600_lam3 --out r.json
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np
import torch

from .rska import Solver

# name: (m, n, s, lambda, eta, noise, iterations, what the figure sweeps)
SETTINGS = {
    # method comparisons (Sec. 5, the first five figures)
    "compare_100x20": dict(m=100, n=20, s=10, lam=1.0, eta=11, noise=0.0, K=2000),
    "compare_100x200": dict(m=100, n=200, s=10, lam=1.0, eta=11, noise=0.0, K=2000),
    "compare_100x500": dict(m=100, n=500, s=10, lam=3.0, eta=11, noise=0.0, K=4000),
    "compare_200x600": dict(m=200, n=600, s=10, lam=3.0, eta=21, noise=0.0, K=4000),
    "compare_300x300": dict(m=300, n=300, s=10, lam=3.0, eta=31, noise=0.0, K=4000),
    # the effect of eta (v2), Sec. 5.1
    "eta_200x600_lam0.01": dict(m=200, n=600, s=10, lam=0.01, eta=None, noise=0.0, K=2000),
    "eta_200x600_lam3": dict(m=200, n=600, s=10, lam=3.0, eta=None, noise=0.0, K=4000),
    "eta_100x10_lam0.01": dict(m=100, n=10, s=10, lam=0.01, eta=None, noise=0.0, K=1000),
    "eta_100x10_lam3": dict(m=100, n=10, s=10, lam=3.0, eta=None, noise=0.0, K=2000),
    # the effect of alpha (v2), Sec. 5.2
    "alpha_200x600": dict(m=200, n=600, s=10, lam=0.1, eta=8, noise=0.0, K=2000),
    "alpha_eta_100x10": dict(m=100, n=10, s=10, lam=6.0, eta=None, noise=0.0, K=100),
    # the effect of lambda, Sec. 5.3
    "lambda_200x600": dict(m=200, n=600, s=10, lam=None, eta=21, noise=0.0, K=1000),
    # noisy right-hand sides, Sec. 5.4 (relative noise level 0.1)
    "noise_100x100": dict(m=100, n=100, s=10, lam=1.0, eta=11, noise=0.1, K=2000),
    "noise_500x100": dict(m=500, n=100, s=10, lam=1.0, eta=11, noise=0.1, K=2000),
    "noise_100x500": dict(m=100, n=500, s=10, lam=1.0, eta=11, noise=0.1, K=2000),
}

VARIANTS = ("rk", "rsk", "v1", "v2", "v3", "v4")


def _problem(m, n, s, seed, noise):
    from synth import gaussian_problem
    return gaussian_problem(m, n, s, seed=seed, noise=noise)


def run_curve(A, b, xhat, n, lam, eta, t, seed, K, check_every, weights=None, couple=False):
    """One run from x_0 = 0: (iterations, relative residuals, relative errors),
    checked every ``check_every`` iterations (and at 0)."""
    dev = torch.device("cuda")
    with Solver(A, b, lam, eta, t, seed, n=n) as sol:
        if weights is not None:
            sol.set_weights(torch.from_numpy(weights).to(dev), couple=couple)
        its, rr, re = [0], [], []
        r0, e0 = sol.metrics(xhat)
        rr.append(r0)
        re.append(e0)
        done = 0
        while done < K:
            step = min(check_every, K - done)
            sol.solve(step)
            done += step
            r, e = sol.metrics(xhat)
            its.append(done)
            rr.append(r)
            re.append(e)
    return np.array(its), np.array(rr), np.array(re)


def _variant_params(variant, lam, eta, sigma2, fro2):
    """(lambda, eta, t, weights-mode) of a variant; weights-mode None, 'v3' or 'v4'."""
    if variant == "rk":
        return 0.0, 1, 1.0, None
    if variant == "rsk":
        return lam, 1, 1.0, None
    if variant == "v1":
        return lam, eta, 1.0, None
    if variant == "v2":
        return lam, eta, eta / (1.0 + (eta - 1) * sigma2 / fro2), None
    if variant in ("v3", "v4"):
        return lam, eta, 1.0, variant
    raise ValueError(variant)


def run_setting(name, trials=5, scale=1, variants=("rk", "rsk", "v2"), etas=(1, 2, 4, 8, 16, 32),
                alphas=None, lambdas=(0.1, 0.5, 1.0, 2.0, 5.0), check_every=None, K=None,
                seed=0):
    """Run one named setting; returns a JSON-able dict of mean/std curves per
    run label (variant, eta, alpha or lambda, by what the setting sweeps)."""
    cfg = dict(SETTINGS[name])
    m, n, s = cfg["m"] * scale, cfg["n"] * scale, cfg["s"] * scale
    K = K or cfg["K"]
    check_every = check_every or max(1, K // 50)
    dev = torch.device("cuda")
    runs = {}
    for tr in range(trials):
        p = _problem(m, n, s, seed=10_000 * (seed + 1) + tr, noise=cfg["noise"])
        A = torch.from_numpy(p.A).to(dev)
        b = torch.from_numpy(p.b).to(dev)
        xh = torch.from_numpy(p.xhat.astype(np.float32)).to(dev)
        with Solver(A, b, 1.0, 1, 1.0, 0, n=n) as probe:
            sigma2, fro2, _ = probe.sigma_max2(100, tr)
        w = np.random.default_rng(tr + 7).uniform(0.0, 1.0, m).astype(np.float32) + 1e-3
        labels = []
        if cfg["eta"] is None and alphas is None:          # eta sweep (v2)
            for e in etas:
                labels.append((f"v2_eta{e}", "v2", cfg["lam"], e, None))
        elif cfg["eta"] is None:                           # alpha x eta grid (v2)
            for e in etas:
                for a in alphas:
                    labels.append((f"eta{e}_alpha{a:g}", "alpha", cfg["lam"], e, a))
        elif cfg["lam"] is None:                           # lambda sweep: RSK vs v2
            for lam in lambdas:
                for v in ("rsk", "v2"):
                    labels.append((f"{v}_lam{lam:g}", v, lam, cfg["eta"], None))
        elif alphas is not None:                           # alpha sweep at fixed eta
            for a in alphas:
                labels.append((f"alpha{a:g}", "alpha", cfg["lam"], cfg["eta"], a))
        else:                                              # method comparison
            for v in variants:
                labels.append((v, v, cfg["lam"], cfg["eta"], None))
        for label, v, lam, eta, alpha in labels:
            if v == "alpha":
                lam_r, eta_r, t_r, wm = lam, eta, alpha, None
            else:
                lam_r, eta_r, t_r, wm = _variant_params(v, lam, eta, sigma2, fro2)
            its, rr, re = run_curve(A, b, xh, n, lam_r, eta_r, t_r, 1000 + tr, K, check_every,
                                    weights=w if wm else None, couple=(wm == "v4"))
            runs.setdefault(label, []).append((its, rr, re))
    out = {"setting": name, "m": m, "n": n, "s": s, "noise": cfg["noise"], "K": K,
           "check_every": check_every, "trials": trials, "runs": {}}
    for label, lst in runs.items():
        its = lst[0][0]
        rr = np.stack([x[1] for x in lst])
        re = np.stack([x[2] for x in lst])
        out["runs"][label] = {
            "iterations": its.tolist(),
            "residual_mean": rr.mean(0).tolist(), "residual_std": rr.std(0).tolist(),
            "error_mean": re.mean(0).tolist(), "error_std": re.std(0).tolist()}
    return out


def iterations_to(curve, tol, key="error_mean"):
    """First checked iteration at which the mean curve is <= tol (None if never)."""
    for it, v in zip(curve["iterations"], curve[key]):
        if v is not None and not math.isnan(v) and v <= tol:
            return it
    return None


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--setting", required=True, choices=sorted(SETTINGS))
    ap.add_argument("--trials", type=int, default=5)
    ap.add_argument("--scale", type=int, default=1)
    ap.add_argument("--variants", default="rk,rsk,v1,v2,v3,v4")
    ap.add_argument("--etas", default="1,2,4,8,16,32")
    ap.add_argument("--alphas", default=None)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    res = run_setting(args.setting, trials=args.trials, scale=args.scale,
                      variants=tuple(args.variants.split(",")),
                      etas=tuple(int(e) for e in args.etas.split(",")),
                      alphas=(tuple(float(a) for a in args.alphas.split(","))
                              if args.alphas else None),
                      K=args.iters)
    text = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    for label, c in res["runs"].items():
        print(f"{label:24s} final residual {c['residual_mean'][-1]:.3e}  "
              f"error {c['error_mean'][-1]:.3e}", file=sys.stderr)
    return 0


if __name__ == "__main__":
    sys.exit(main())
