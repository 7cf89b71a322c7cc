"""FP64 CPU oracle for randomized sparse Kaczmarz with averaging (RSKA).

TEST INFRASTRUCTURE ONLY.  Tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library and its
Python binding never do.  The oracle is ``rska_oracle.c`` (plain C, FP64,
single-threaded, ``-O2 -ffp-contract=off``) behind ctypes; this module only
marshals arrays.  It shares no code with ``paper_2203_10838_gb300``.

What each function follows in the paper (Tondji & Lorenz, arXiv 2203.10838):

* ``philox4x32_10`` -- the counter-based generator of Salmon et al. (SC'11)
  used to draw tau_k (Algorithm 1: "eta indices sampled").
* ``row_norms``     -- ||a_i||^2 of Definition 1 (matrix D), in the canonical
  summation order of the index contract.
* ``alias_build``   -- Walker/Vose table for p_i = ||a_i||^2 / ||A||_F^2
  (Sec. 5, variants v1/v2).
* ``sample``        -- tau_k with replacement (eq. rska, Algorithm 1).
* ``rska_fixed`` / ``rska`` -- eq. (rska) / Algorithm 1 with w_i = t, or
  t w_i for given row weights (Sec. 5, variants v3/v4).
* ``linearized_bregman`` -- the full-gradient limit eta -> infinity of
  eq. (rska) (Sec. 4 remarks), step by step.
* ``sigma_max2`` / ``alpha_star`` -- sigma_max(A)^2 (the largest eigenvalue
  of A^T A, a library eigensolver in FP64) and the step alpha^*(eta) of
  Corollary 1 (uniform weights).
* ``rska_mrhs``     -- eq. (rska) on every right-hand side b_j of a shared A
  with one index sequence (the matrix form A^T M_k (A x - b) of Sec. 3 per
  column).
* ``metrics``       -- relative residual and error of Sec. 5.
* ``unrolled_grad`` -- reverse-mode gradient of K unrolled iterations of
  eq. (rska) (the paper has no gradient; this differentiates it as written).

Parity status: every function above is pinned by tests under ``tests/``
(``test_oracle_*.py``); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rska_oracle.c")
_LIB_PATH = os.path.join(_HERE, "librska_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/librska_oracle.so``."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
             "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32, u32, u64, f64 = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                               ctypes.c_uint64, ctypes.c_double)
    lib.orc_philox4x32_10.argtypes = [P, P, P]
    lib.orc_philox4x32_10.restype = None
    lib.orc_row_norms.argtypes = [P, i64, i64, i64, P]
    lib.orc_row_norms.restype = None
    lib.orc_alias_build.argtypes = [P, i64, P, P]
    lib.orc_alias_build.restype = ctypes.c_int
    lib.orc_sample.argtypes = [P, P, i64, u64, u32, i64, i64, i32, P]
    lib.orc_sample.restype = None
    lib.orc_rska_fixed.argtypes = [P, i64, i64, i64, P, P, f64, f64, i32, P, i64, P]
    lib.orc_rska_fixed.restype = ctypes.c_int
    lib.orc_rska_fixed_weighted.argtypes = [P, i64, i64, i64, P, P, P, f64, f64, i32, P, i64,
                                            P]
    lib.orc_rska_fixed_weighted.restype = ctypes.c_int
    lib.orc_rska_sampled.argtypes = [P, i64, i64, i64, P, P, P, P, f64, f64, i32, u64, u32,
                                     i64, i64, P]
    lib.orc_rska_sampled.restype = ctypes.c_int
    lib.orc_metrics.argtypes = [P, i64, i64, i64, P, P, f64, P, P, P]
    lib.orc_metrics.restype = None
    lib.orc_unrolled_grad.argtypes = [P, i64, i64, i64, P, P, f64, f64, i32, P, i64, P, P, P,
                                      P, P]
    lib.orc_unrolled_grad.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_A(A):
    """A as a C-contiguous float32 matrix plus its leading dimension."""
    A = np.asarray(A)
    if A.dtype != np.float32:
        A = A.astype(np.float32)
    if not A.flags.c_contiguous:
        A = np.ascontiguousarray(A)
    return A, A.shape[1]


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def row_norms(A) -> np.ndarray:
    A, lda = _as_A(A)
    m, n = A.shape
    nu = np.zeros(m, dtype=np.float64)
    _load().orc_row_norms(_ptr(A), m, n, lda, _ptr(nu))
    return nu


def alias_build(nu):
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    m = nu.shape[0]
    thr = np.zeros(max(m, 1), dtype=np.uint32)
    alias = np.zeros(max(m, 1), dtype=np.int32)
    rc = _load().orc_alias_build(_ptr(nu), m, _ptr(thr), _ptr(alias))
    if rc != 0:
        raise ValueError(f"alias_build failed ({rc}): rows must have finite nonzero norms")
    return thr[:m], alias[:m]


def sample(thr, alias, seed: int, eta: int, k0: int, K: int, problem: int = 0) -> np.ndarray:
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    alias = np.ascontiguousarray(alias, dtype=np.int32)
    out = np.zeros(K * eta, dtype=np.int32)
    _load().orc_sample(_ptr(thr), _ptr(alias), thr.shape[0], seed, problem, k0, K, eta, _ptr(out))
    return out.reshape(K, eta)


def rska_fixed(A, b, lam: float, t: float, eta: int, tau, z0=None, nu=None,
               w=None) -> np.ndarray:
    """K = len(tau) iterations of eq. (rska) with the given index sequence.

    tau has shape (K, eta).  w (optional, m entries) is the diagonal of the
    weight matrix W: row i's step is scaled by t * w_i (Sec. 5, v3/v4 with
    t = 1).  Returns the dual iterate z_K (x_K = S_lam(z_K)).
    """
    A, lda = _as_A(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    nu = row_norms(A) if nu is None else np.ascontiguousarray(nu, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.int32).reshape(-1, eta)
    if tau.size and (tau.min() < 0 or tau.max() >= m):
        raise ValueError("index out of range")
    z = np.zeros(n, dtype=np.float64) if z0 is None else np.array(z0, dtype=np.float64)
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (m,):
            raise ValueError("w must have one entry per row")
        rc = _load().orc_rska_fixed_weighted(_ptr(A), m, n, lda, _ptr(b), _ptr(nu), _ptr(w),
                                             lam, t, eta, _ptr(tau), tau.shape[0], _ptr(z))
        if rc != 0:
            raise ValueError(f"rska_fixed_weighted failed ({rc})")
        return z
    rc = _load().orc_rska_fixed(_ptr(A), m, n, lda, _ptr(b), _ptr(nu), lam, t, eta, _ptr(tau),
                                tau.shape[0], _ptr(z))
    if rc != 0:
        raise ValueError(f"rska_fixed failed ({rc})")
    return z


def rska(A, b, lam: float, eta: int, t: float, seed: int, K: int, k0: int = 0, z0=None,
         problem: int = 0, tables=None) -> np.ndarray:
    """K iterations of Algorithm 1 drawing tau_k, k = k0..k0+K-1, by the index
    contract.  Returns z_{k0+K}."""
    A, lda = _as_A(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    if tables is None:
        nu = row_norms(A)
        thr, alias = alias_build(nu)
    else:
        nu, thr, alias = tables
    z = np.zeros(n, dtype=np.float64) if z0 is None else np.array(z0, dtype=np.float64)
    rc = _load().orc_rska_sampled(_ptr(A), m, n, lda, _ptr(b), _ptr(nu), _ptr(thr), _ptr(alias),
                                  lam, t, eta, seed, problem, k0, K, _ptr(z))
    if rc != 0:
        raise ValueError(f"rska failed ({rc})")
    return z


def rska_mrhs(A, B, lam: float, t: float, eta: int, tau, nu=None, rows=None) -> np.ndarray:
    """Shared-A multi-right-hand-side RSKA: for each right-hand side b_j
    (row j of B), K = len(tau) iterations of eq. (rska) on (A, b_j) with the
    one index sequence tau shared by all j -- the update A^T M_k (A x - b) of
    Sec. 3 applied to every column of X at once.  Returns Z with one row z_j
    per requested j (``rows``, default all)."""
    A, lda = _as_A(A)
    nu = row_norms(A) if nu is None else np.ascontiguousarray(nu, dtype=np.float64)
    B = np.asarray(B)
    rows = range(B.shape[0]) if rows is None else rows
    return np.stack([rska_fixed(A, B[j], lam, t, eta, tau, nu=nu) for j in rows])


def sigma_max2(A) -> float:
    """sigma_max(A)^2: the largest eigenvalue of A^T A (or A A^T, the smaller
    of the two) formed in FP64 from the FP32 values."""
    A = np.asarray(A, dtype=np.float64)
    G = A.T @ A if A.shape[1] <= A.shape[0] else A @ A.T
    return float(np.linalg.eigvalsh(G)[-1])


def alpha_star(eta: int, sigma2: float, fro2: float) -> float:
    """alpha^* = eta / (1 + (eta - 1) sigma_max^2 / ||A||_F^2), the uniform
    weight of Corollary 1 that maximises the rate bound L(alpha)."""
    return eta / (1.0 + (eta - 1) * sigma2 / fro2)


def linearized_bregman(A, b, lam: float, step: float, K: int, z0=None) -> np.ndarray:
    """K iterations of the linearized Bregman method (the remark on its rate
    in Sec. 4): z <- z - step A^T (A x - b), x = S_lam(z), in FP64 on the
    FP32 values of A.  Returns z_K."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    z = np.zeros(A.shape[1]) if z0 is None else np.array(z0, dtype=np.float64)
    for _ in range(K):
        x = soft_shrink(z, lam)
        z = z - step * (A.T @ (A @ x - b))
    return z


def soft_shrink(z, lam: float) -> np.ndarray:
    """S_lam(z) = max(|z| - lam, 0) sign(z) (Sec. 1.1)."""
    z = np.asarray(z, dtype=np.float64)
    return np.sign(z) * np.maximum(np.abs(z) - lam, 0.0)


def metrics(A, b, z, lam: float, xhat=None):
    A, lda = _as_A(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    rr = ctypes.c_double(0.0)
    re = ctypes.c_double(float("nan"))
    xh = None
    if xhat is not None:
        xh = np.ascontiguousarray(xhat, dtype=np.float64)
    _load().orc_metrics(_ptr(A), m, n, lda, _ptr(b), _ptr(z), lam,
                        _ptr(xh) if xh is not None else None, ctypes.byref(rr), ctypes.byref(re))
    return rr.value, (re.value if xh is not None else None)


def unrolled_grad(A, b, lam: float, t: float, eta: int, tau, xhat, nu=None):
    """Loss 1/2||x_K - xhat||^2 of K = len(tau) unrolled iterations and its
    gradient with respect to b, lambda and t.  Returns (loss, gb, glam, gt)."""
    A, lda = _as_A(A)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    nu = row_norms(A) if nu is None else np.ascontiguousarray(nu, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.int32).reshape(-1, eta)
    xhat = np.ascontiguousarray(xhat, dtype=np.float64)
    loss = ctypes.c_double(0.0)
    glam = ctypes.c_double(0.0)
    gt = ctypes.c_double(0.0)
    gb = np.zeros(m, dtype=np.float64)
    rc = _load().orc_unrolled_grad(_ptr(A), m, n, lda, _ptr(b), _ptr(nu), lam, t, eta, _ptr(tau),
                                   tau.shape[0], _ptr(xhat), ctypes.byref(loss), _ptr(gb),
                                   ctypes.byref(glam), ctypes.byref(gt))
    if rc != 0:
        raise ValueError(f"unrolled_grad failed ({rc})")
    return loss.value, gb, glam.value, gt.value
