"""Seeded synthetic RSKA problems (inputs only; no solver arithmetic here).

Shared by the tests, the benchmark, the oracle side and the CUDA side, which
otherwise share nothing.  The recipe follows the paper's Sec. 5 (Tondji &
Lorenz, arXiv 2203.10838): A has i.i.d. N(0, 1) entries, the solution xhat has
s nonzeros at positions drawn uniformly without replacement with N(0, 1)
values, b = A xhat, and a noisy right-hand side adds a vector drawn uniformly
on the sphere of radius ell * ||A xhat|| (the "relative noise level" ell of
the noisy-case experiments).  Everything comes from numpy's PCG64 generator
seeded by the caller.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    A: np.ndarray       # (m, lda) float32, row-major; columns >= n are padding (zeros)
    b: np.ndarray       # (m,) float32 right-hand side handed to both sides
    xhat: np.ndarray    # (n,) float64 planted sparse solution
    n: int
    b64: np.ndarray     # (m,) float64 right-hand side before rounding to float32

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def lda(self) -> int:
        return self.A.shape[1]


def round_up(v: int, k: int) -> int:
    return ((v + k - 1) // k) * k


def gaussian_problem(m: int, n: int, s: int, seed: int, noise: float = 0.0,
                     lda: int | None = None, scale: float = 1.0) -> Problem:
    """A ~ N(0, scale^2) i.i.d. (float32), s-sparse xhat, b = A xhat (+ noise).

    ``lda`` defaults to n rounded up to a multiple of 4 (16-byte rows); padding
    columns are zero.  ``noise`` is the relative level ell: b gets
    ell * ||A xhat|| * g / ||g|| added with g ~ N(0, I_m).
    """
    if lda is None:
        lda = round_up(n, 4)
    rng = np.random.default_rng(seed)
    A = np.zeros((m, lda), dtype=np.float32)
    A[:, :n] = rng.standard_normal((m, n), dtype=np.float32)
    if scale != 1.0:
        A[:, :n] *= np.float32(scale)
    xhat = np.zeros(n, dtype=np.float64)
    s = min(s, n)
    support = rng.choice(n, size=s, replace=False)
    xhat[support] = rng.standard_normal(s)
    # b = A xhat in FP64; only the support columns of A contribute
    b64 = A[:, support].astype(np.float64) @ xhat[support]
    if noise > 0.0:
        g = rng.standard_normal(m)
        b64 = b64 + noise * np.linalg.norm(b64) * g / np.linalg.norm(g)
    return Problem(A=A, b=b64.astype(np.float32), xhat=xhat, n=n, b64=b64)


def batched_sizes(P: int, seed: int, m_lo: int = 200, m_hi: int = 4000):
    """m_p log-uniform in [m_lo, m_hi], n_p = m_p/2 rounded to a multiple of 8."""
    rng = np.random.default_rng(seed)
    logm = rng.uniform(np.log(m_lo), np.log(m_hi), size=P)
    m = np.clip(np.rint(np.exp(logm)).astype(np.int64), m_lo, m_hi)
    n = np.maximum(8, np.rint(m / 2.0 / 8.0).astype(np.int64) * 8)
    return m, n


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32 holding exactly the bfloat16 value."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def pack_batch(problems):
    """Concatenate Problems for the batched interface: returns (A_flat, a_off,
    m, n, lda, b_flat, b_off) with every A_p starting on a 16-byte boundary."""
    a_off, b_off, m, n, lda = [], [], [], [], []
    total_a = total_b = 0
    for pr in problems:
        a_off.append(total_a)
        b_off.append(total_b)
        m.append(pr.m)
        n.append(pr.n)
        lda.append(pr.lda)
        total_a += round_up(pr.m * pr.lda, 4)
        total_b += pr.m
    A = np.zeros(total_a, dtype=np.float32)
    b = np.zeros(total_b, dtype=np.float32)
    for pr, ao, bo in zip(problems, a_off, b_off):
        A[ao:ao + pr.m * pr.lda] = pr.A.ravel()
        b[bo:bo + pr.m] = pr.b
    as64 = lambda v: np.asarray(v, dtype=np.int64)
    return A, as64(a_off), as64(m), as64(n), as64(lda), b, as64(b_off)


def batched_problem_set(P: int, seed: int, m_lo: int = 200, m_hi: int = 4000, threads: int = 0,
                        subset=None):
    """The batched workload of independent Gaussian systems, generated straight
    into packed arrays: m_p log-uniform in [m_lo, m_hi], n_p = m_p / 2 rounded
    to a multiple of 8, s_p = n_p / 20, problem p drawn exactly as
    gaussian_problem(m_p, n_p, s_p, seed + 1 + p).  Returns (A_flat, a_off, m,
    n, lda, b_flat, b_off, xhats).  With ``subset`` (problem indices of the
    P-problem set) only those problems are generated and packed, in the given
    order, each with exactly the values it has in the whole set."""
    import concurrent.futures
    import os
    ms, ns = batched_sizes(P, seed, m_lo, m_hi)
    ids = np.arange(P, dtype=np.int64) if subset is None else np.asarray(subset, dtype=np.int64)
    ms, ns = ms[ids], ns[ids]
    P = len(ids)
    ldas = np.array([round_up(int(v), 4) for v in ns], dtype=np.int64)
    sizes = np.array([round_up(int(mm) * int(ll), 4) for mm, ll in zip(ms, ldas)], dtype=np.int64)
    a_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(ms)[:-1]]).astype(np.int64)
    A = np.empty(int(sizes.sum()), dtype=np.float32)
    b = np.empty(int(ms.sum()), dtype=np.float32)
    xhats = [None] * P

    def make(p):
        m, n, lda = int(ms[p]), int(ns[p]), int(ldas[p])
        view = A[a_off[p]:a_off[p] + m * lda].reshape(m, lda)
        rng = np.random.default_rng(seed + 1 + int(ids[p]))
        if lda == n:
            rng.standard_normal(out=view, dtype=np.float32)
        else:
            view[:, :n] = rng.standard_normal((m, n), dtype=np.float32)
            view[:, n:] = 0.0
        s = max(1, n // 20)
        xhat = np.zeros(n, dtype=np.float64)
        support = rng.choice(n, size=s, replace=False)
        xhat[support] = rng.standard_normal(s)
        b[b_off[p]:b_off[p] + m] = (view[:, support].astype(np.float64) @ xhat[support])
        xhats[p] = xhat

    workers = threads or min(32, os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        list(ex.map(make, range(P)))
    return A, a_off, ms.astype(np.int64), ns.astype(np.int64), ldas, b, b_off, xhats


@dataclass
class MultiProblem:
    A16: np.ndarray     # (m, lda) uint16: the BF16 bit patterns of A (padding columns zero)
    A: np.ndarray       # (m, lda) float32 holding exactly the same BF16 values
    B: np.ndarray       # (R, m) float32, row j = b_j
    B64: np.ndarray     # (R, m) float64 right-hand sides before rounding to float32
    Xhat: np.ndarray    # (R, n) float64 planted sparse solutions
    n: int

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def R(self) -> int:
        return self.B.shape[0]


def multi_rhs_problem(m: int, n: int, R: int, s: int, seed: int, scale: float | None = None,
                      lda: int | None = None) -> MultiProblem:
    """Shared-A multi-right-hand-side workload: A i.i.d. N(0, scale^2) (scale
    defaults to 1/sqrt(n)) rounded to BF16, R planted solutions xhat_j with s
    nonzeros N(0, 1) at uniformly drawn positions, and b_j = A_bf16 xhat_j
    computed in FP64 from the BF16 values (so xhat_j solves the stored
    system exactly) then rounded to float32.  ``lda`` defaults to n rounded up
    to a multiple of 8; padding columns are zero."""
    if lda is None:
        lda = round_up(n, 8)
    if scale is None:
        scale = 1.0 / np.sqrt(n)
    rng = np.random.default_rng(seed)
    A = np.zeros((m, lda), dtype=np.float32)
    A[:, :n] = rng.standard_normal((m, n), dtype=np.float32) * np.float32(scale)
    A = bf16_round(A)
    A16 = (A.view(np.uint32) >> 16).astype(np.uint16)
    s = min(s, n)
    Xhat = np.zeros((R, n), dtype=np.float64)
    for j in range(R):
        support = rng.choice(n, size=s, replace=False)
        Xhat[j, support] = rng.standard_normal(s)
    B64 = np.empty((R, m), dtype=np.float64)
    XT = Xhat.T.copy()
    for r0 in range(0, m, 2048):
        B64[:, r0:r0 + 2048] = (A[r0:r0 + 2048, :n].astype(np.float64) @ XT).T
    return MultiProblem(A16=A16, A=A, B=B64.astype(np.float32), B64=B64, Xhat=Xhat, n=n)
