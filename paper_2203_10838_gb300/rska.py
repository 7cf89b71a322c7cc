"""Thin Python binding of the librska C ABI (include/rska.h) over torch tensors.

Argument marshalling only: torch provides device memory and the CUDA stream;
every step of RSKA (eq. rska, Algorithm 1 of Tondji & Lorenz, arXiv
2203.10838) runs in librska's kernels.  Names mirror the C entry points.
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import check, lib

QUERY = {"grid": 0, "threads": 1, "rows_resident": 2, "w4max": 3, "smem": 4, "rreg": 5,
         "kernel": 6, "setup_alloc_us": 7, "setup_norms_us": 8, "setup_alias_us": 9,
         "setup_total_us": 10}
OPTION = {"grid": 0, "watchdog_us": 1, "kernel": 2}
KERNEL = {"auto": 0, "column": 1, "rows": 2, "small": 3}


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("librska takes device tensors")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One RSKA problem: rska_setup on construction, rska_destroy on close().

    A: (m, lda) float32 tensor, row-major, lda a multiple of 4; the first n
    columns are the matrix (n defaults to lda).  b: (m,) float32 tensor.  CUDA
    tensors are borrowed by the library and kept alive here; CPU tensors are
    copied by the library (rska_setup_host, overlapped with the setup when
    pinned).
    """

    def __init__(self, A: torch.Tensor, b: torch.Tensor, lam: float, eta: int, t: float,
                 seed: int, n: int | None = None, stream: torch.cuda.Stream | None = None):
        if A.dtype != torch.float32 or b.dtype != torch.float32:
            raise ValueError("A and b must be float32")
        if A.dim() != 2 or b.dim() != 1 or b.shape[0] != A.shape[0]:
            raise ValueError("A must be (m, lda) and b (m,)")
        self.A, self.b = A, b
        self.m, self.lda = A.shape
        self.n = self.lda if n is None else int(n)
        self.eta, self.lam, self.t, self.seed = int(eta), float(lam), float(t), int(seed)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        if A.is_cuda:
            self.device = A.device
            check(lib().rska_setup(ctypes.byref(h), _dptr(A), self.m, self.n, self.lda,
                                   _dptr(b), self.lam, self.eta, self.t, self.seed,
                                   _stream_ptr(self.stream)), "rska_setup")
        else:
            # host tensors: rska_setup_host copies them (overlapped with the
            # row norms when they are pinned); the library owns the copies
            if b.is_cuda or not A.is_contiguous() or not b.is_contiguous():
                raise ValueError("host A and b must both be contiguous CPU tensors")
            self.device = self.stream.device
            check(lib().rska_setup_host(ctypes.byref(h), ctypes.c_void_p(A.data_ptr()), self.m,
                                        self.n, self.lda, ctypes.c_void_p(b.data_ptr()),
                                        self.lam, self.eta, self.t, self.seed,
                                        _stream_ptr(self.stream)), "rska_setup_host")
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().rska_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points -----------------------------------------------------
    def load_host(self, A: torch.Tensor, b: torch.Tensor):
        """rska_load_host: a new problem of this context's shape from host
        tensors (float32, contiguous; pinned memory overlaps the copy with the
        row norms), reusing the context's device memory; z = 0, k = 0."""
        if A.is_cuda or b.is_cuda or A.dtype != torch.float32 or b.dtype != torch.float32:
            raise ValueError("load_host takes float32 CPU tensors")
        if tuple(A.shape) != (self.m, self.lda) or tuple(b.shape) != (self.m,):
            raise ValueError("A and b must have the shape of the context's problem")
        if not A.is_contiguous() or not b.is_contiguous():
            raise ValueError("A and b must be contiguous")
        self.A, self.b = A, b
        check(lib().rska_load_host(self._h, ctypes.c_void_p(A.data_ptr()),
                                   ctypes.c_void_p(b.data_ptr())), "rska_load_host")

    def solve(self, K: int):
        check(lib().rska_solve(self._h, int(K)), "rska_solve")

    def solve_until(self, max_iters: int, check_every: int, tol: float,
                    xhat: torch.Tensor | None = None):
        it = ctypes.c_int64()
        met = ctypes.c_double()
        check(lib().rska_solve_until(self._h, int(max_iters), int(check_every), float(tol),
                                     _dptr(xhat), ctypes.byref(it), ctypes.byref(met)),
              "rska_solve_until")
        return it.value, met.value

    def get_x(self):
        x = torch.empty(self.n, dtype=torch.float32, device=self.device)
        z = torch.empty(self.n, dtype=torch.float32, device=self.device)
        check(lib().rska_get_x(self._h, _dptr(x), _dptr(z)), "rska_get_x")
        return x, z

    def set_state(self, z: torch.Tensor, k: int):
        check(lib().rska_set_state(self._h, _dptr(z), int(k)), "rska_set_state")

    @property
    def iteration(self) -> int:
        k = ctypes.c_int64()
        check(lib().rska_iteration(self._h, ctypes.byref(k)), "rska_iteration")
        return k.value

    def get_indices(self, k0: int, K: int) -> torch.Tensor:
        out = torch.empty((K, self.eta), dtype=torch.int32, device=self.device)
        check(lib().rska_get_indices(self._h, int(k0), int(K), _dptr(out)), "rska_get_indices")
        return out

    def get_tables(self):
        nu = torch.empty(self.m, dtype=torch.float64, device=self.device)
        thr = torch.empty(self.m, dtype=torch.int32, device=self.device)
        alias = torch.empty(self.m, dtype=torch.int32, device=self.device)
        check(lib().rska_get_tables(self._h, _dptr(nu), _dptr(thr), _dptr(alias)),
              "rska_get_tables")
        return nu, thr, alias

    def metrics(self, xhat: torch.Tensor | None = None):
        rr = ctypes.c_double()
        re = ctypes.c_double(float("nan"))
        check(lib().rska_metrics(self._h, _dptr(xhat), ctypes.byref(rr), ctypes.byref(re)),
              "rska_metrics")
        return rr.value, (re.value if xhat is not None else None)

    def reset(self):
        check(lib().rska_reset(self._h), "rska_reset")

    def query(self, what: str) -> int:
        v = ctypes.c_int64()
        check(lib().rska_query(self._h, QUERY[what], ctypes.byref(v)), "rska_query")
        return v.value

    def set_option(self, what: str, value: int):
        check(lib().rska_set_option(self._h, OPTION[what], int(value)), "rska_set_option")

    def sigma_max2(self, iters: int = 50, seed: int = 0):
        """(sigma_max(A)^2 estimate, ||A||_F^2, alpha^*(eta)) by power
        iteration on A^T A (Corollary 1)."""
        s2, f2, al = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().rska_sigma_max2(self._h, int(iters), int(seed), ctypes.byref(s2),
                                    ctypes.byref(f2), ctypes.byref(al)), "rska_sigma_max2")
        return s2.value, f2.value, al.value

    def linearized_bregman(self, K: int, step: float):
        """K iterations of z -= step A^T (A x - b), x = S_lam(z) (the eta ->
        infinity limit of RSKA; the paper's step is 1/sigma_max(A)^2)."""
        check(lib().rska_linearized_bregman(self._h, int(K), float(step)),
              "rska_linearized_bregman")

    def set_weights(self, w=None, couple: bool = False):
        """Row weights w_i of eq. (rska) (Sec. 5, v3: couple=False keeps
        p_i ~ ||a_i||^2; v4: couple=True samples p_i ~ ||a_i||^2 / w_i).
        w: float32 CUDA tensor of m entries, finite and > 0, or None for
        uniform weights."""
        ptr = None
        if w is not None:
            if (not w.is_cuda or w.dtype != torch.float32 or w.dim() != 1
                    or w.shape[0] != self.m or not w.is_contiguous()):
                raise ValueError("w must be a contiguous float32 CUDA vector of m entries")
            ptr = ctypes.c_void_p(w.data_ptr())
        check(lib().rska_set_weights(self._h, ptr, 1 if couple else 0), "rska_set_weights")


def rska_setup(A, b, lam, eta, t, seed, n=None, stream=None) -> Solver:
    return Solver(A, b, lam, eta, t, seed, n=n, stream=stream)


def rska_solve(solver: Solver, K: int):
    solver.solve(K)


def rska_get_x(solver: Solver):
    return solver.get_x()


def rska_destroy(solver: Solver):
    solver.close()


def rska_solve_noalloc(A: torch.Tensor, b: torch.Tensor, lam: float, eta: int, t: float,
                       seed: int, K: int, n: int | None = None, stream=None):
    """One-shot solve that allocates no device memory inside the library (its
    working memory is a fixed device array); returns (x, z).  The output
    tensors are allocated here by torch, before the call."""
    if A.dtype != torch.float32 or b.dtype != torch.float32:
        raise ValueError("A and b must be float32")
    m, lda = A.shape
    n = lda if n is None else int(n)
    x = torch.empty(n, dtype=torch.float32, device=A.device)
    z = torch.empty(n, dtype=torch.float32, device=A.device)
    check(lib().rska_solve_noalloc(_dptr(A), m, n, lda, _dptr(b), float(lam), int(eta), float(t),
                                   int(seed), int(K), _dptr(x), _dptr(z), _stream_ptr(stream)),
          "rska_solve_noalloc")
    return x, z


def rska_probe_l2_read(buf: torch.Tensor, reps: int, ctas: int, sink: torch.Tensor,
                       stream=None):
    """Launch the L2 read-bandwidth probe over the device tensor `buf`
    (asynchronous on `stream`); the caller times it."""
    check(lib().rska_probe_l2_read(_dptr(buf), buf.numel() * buf.element_size(), int(reps),
                                   int(ctas), _dptr(sink), _stream_ptr(stream)),
          "rska_probe_l2_read")


class BatchSolver:
    """Many independent problems in one persistent launch (rska_batch_*).

    A: packed float32 CUDA tensor holding every A_p at element offset a_off[p]
    (row-major, leading dimension lda[p]); b: packed float32 CUDA tensor with
    b_p at b_off[p].  a_off, m, n, lda, b_off: integer sequences (host).
    """

    def __init__(self, A: torch.Tensor, b: torch.Tensor, a_off, m, n, lda, b_off, lam: float,
                 eta: int, t: float, seed: int, stream=None):
        import numpy as np
        self.A, self.b = A, b
        self.P = len(m)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = A.device
        self._host = [np.ascontiguousarray(v, dtype=np.int64) for v in (a_off, m, n, lda, b_off)]
        ptrs = [ctypes.c_void_p(v.ctypes.data) for v in self._host]
        h = ctypes.c_void_p()
        check(lib().rska_batch_setup(ctypes.byref(h), self.P, _dptr(A), *ptrs[:4], _dptr(b),
                                     ptrs[4], float(lam), int(eta), float(t), int(seed),
                                     _stream_ptr(self.stream)), "rska_batch_setup")
        self._h = h
        self.x_off = np.zeros(self.P + 1, dtype=np.int64)
        check(lib().rska_batch_offsets(self._h, ctypes.c_void_p(self.x_off.ctypes.data)),
              "rska_batch_offsets")

    def close(self):
        if getattr(self, "_h", None):
            lib().rska_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream_ids(self, ids):
        """Index-stream id of each problem (counter word 3 of the index
        contract; default: its position in this batch)."""
        import numpy as np
        arr = np.ascontiguousarray(ids, dtype=np.uint32)
        if arr.shape != (self.P,):
            raise ValueError("one stream id per problem")
        check(lib().rska_batch_set_stream_ids(self._h, ctypes.c_void_p(arr.ctypes.data)),
              "rska_batch_set_stream_ids")

    def solve(self, max_iters: int, tol: float = 0.0, check_every: int = 0):
        check(lib().rska_batch_solve(self._h, int(max_iters), float(tol), int(check_every)),
              "rska_batch_solve")

    def results(self):
        import numpy as np
        it = np.zeros(self.P, dtype=np.int64)
        rr = np.zeros(self.P, dtype=np.float64)
        check(lib().rska_batch_results(self._h, ctypes.c_void_p(it.ctypes.data),
                                       ctypes.c_void_p(rr.ctypes.data)), "rska_batch_results")
        return it, rr

    def get_x(self):
        total = int(self.x_off[-1])
        x = torch.empty(total, dtype=torch.float32, device=self.device)
        z = torch.empty(total, dtype=torch.float32, device=self.device)
        check(lib().rska_batch_get_x(self._h, _dptr(x), _dptr(z)), "rska_batch_get_x")
        return x, z

    def get_tables(self):
        rows = int(sum(int(v) for v in self._host[1]))
        nu = torch.empty(rows, dtype=torch.float64, device=self.device)
        thr = torch.empty(rows, dtype=torch.int32, device=self.device)
        alias = torch.empty(rows, dtype=torch.int32, device=self.device)
        check(lib().rska_batch_get_tables(self._h, _dptr(nu), _dptr(thr), _dptr(alias)),
              "rska_batch_get_tables")
        return nu, thr, alias


MRHS_OPTION = {"terms": 0, "ksplit": 1, "watchdog_us": 2, "graph": 3, "pdl": 4, "form": 5,
               "terms_update": 6, "gather_sched": 7}
MRHS_QUERY = {"k": 0, "ksplit": 1, "n_pad": 2, "eta_pad": 3, "R_pad": 4, "terms": 5, "form": 6,
              "terms_update": 7, "gather_sched": 8, "tuned_code": 9, "tuned_ns": 10,
              "ksplit_used": 11, "pdl": 12}


def decode_schedule(code: int) -> dict:
    """A schedule code of rska_mrhs_tune / rska_tune_candidates as a dict."""
    form = code & 3
    if form == 2:
        return {"form": "persistent", "gather_sched": (code >> 17) & 7}
    return {"form": "staged", "ksplit": (code >> 8) & 0xff, "pdl": (code >> 16) & 1}


def tune_candidates(n: int, R: int, eta: int, num_sms: int) -> list:
    """rska_tune_candidates: the candidate schedule codes (no device work)."""
    count = ctypes.c_int32()
    check(lib().rska_tune_candidates(int(n), int(R), int(eta), int(num_sms), None, 0,
                                     ctypes.byref(count)), "rska_tune_candidates")
    buf = (ctypes.c_int32 * max(1, count.value))()
    check(lib().rska_tune_candidates(int(n), int(R), int(eta), int(num_sms), buf, count.value,
                                     ctypes.byref(count)), "rska_tune_candidates")
    return [int(buf[i]) for i in range(count.value)]


def tune_cache(op: str, key_or_path: str | None = None, code: int = 0, us: float = 0.0):
    """rska_tune_cache: op "get" -> (code, us) or None, "put", "save", "load", "clear"."""
    ops = {"get": 0, "put": 1, "save": 2, "load": 3, "clear": 4}
    c = ctypes.c_int32(int(code))
    u = ctypes.c_double(float(us))
    k = key_or_path.encode() if key_or_path is not None else None
    rc = lib().rska_tune_cache(ops[op], k, ctypes.byref(c), ctypes.byref(u))
    if op == "get":
        return (int(c.value), float(u.value)) if rc == 0 else None
    check(rc, "rska_tune_cache")
MRHS_FORM = {"auto": 0, "staged": 1, "persistent": 2}


class MultiRHS:
    """Shared-A multi-right-hand-side RSKA on the tensor cores (rska_mrhs_*).

    A: (m, lda) torch.bfloat16 CUDA tensor (lda a multiple of 8; the first n
    columns are the matrix, n defaults to lda), borrowed by the library and
    kept alive here.  B: (R, m) float32 CUDA tensor, row j = b_j (copied
    during setup).  Results come back as (R, n) tensors, row j = x_j.
    """

    def __init__(self, A: torch.Tensor, B: torch.Tensor, lam: float, eta: int, t: float,
                 seed: int, n: int | None = None, stream: torch.cuda.Stream | None = None):
        if A.dtype != torch.bfloat16 or B.dtype != torch.float32:
            raise ValueError("A must be bfloat16 and B float32")
        if A.dim() != 2 or B.dim() != 2 or B.shape[1] != A.shape[0]:
            raise ValueError("A must be (m, lda) and B (R, m)")
        self.A = A
        self.m, self.lda = A.shape
        self.R = B.shape[0]
        self.n = self.lda if n is None else int(n)
        self.eta, self.lam, self.t, self.seed = int(eta), float(lam), float(t), int(seed)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = A.device
        h = ctypes.c_void_p()
        check(lib().rska_mrhs_setup(ctypes.byref(h), _dptr(A), self.m, self.n, self.lda, _dptr(B),
                                    self.R, B.shape[1], self.lam, self.eta, self.t, self.seed,
                                    _stream_ptr(self.stream)), "rska_mrhs_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().rska_mrhs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, K: int):
        check(lib().rska_mrhs_solve(self._h, int(K)), "rska_mrhs_solve")

    def get_x(self):
        x = torch.empty((self.R, self.n), dtype=torch.float32, device=self.device)
        z = torch.empty((self.R, self.n), dtype=torch.float32, device=self.device)
        check(lib().rska_mrhs_get_x(self._h, _dptr(x), _dptr(z)), "rska_mrhs_get_x")
        return x, z

    def get_indices(self, k0: int, K: int) -> torch.Tensor:
        out = torch.empty((K, self.eta), dtype=torch.int32, device=self.device)
        check(lib().rska_mrhs_get_indices(self._h, int(k0), int(K), _dptr(out)),
              "rska_mrhs_get_indices")
        return out

    def get_tables(self):
        nu = torch.empty(self.m, dtype=torch.float64, device=self.device)
        thr = torch.empty(self.m, dtype=torch.int32, device=self.device)
        alias = torch.empty(self.m, dtype=torch.int32, device=self.device)
        check(lib().rska_mrhs_get_tables(self._h, _dptr(nu), _dptr(thr), _dptr(alias)),
              "rska_mrhs_get_tables")
        return nu, thr, alias

    def reset(self):
        check(lib().rska_mrhs_reset(self._h), "rska_mrhs_reset")

    def set_option(self, what: str, value: int):
        check(lib().rska_mrhs_set_option(self._h, MRHS_OPTION[what], int(value)),
              "rska_mrhs_set_option")

    def tune(self, iters: int = 64):
        """rska_mrhs_tune: (chosen code, microseconds per iteration)."""
        c = ctypes.c_int32()
        u = ctypes.c_double()
        check(lib().rska_mrhs_tune(self._h, int(iters), ctypes.byref(c), ctypes.byref(u)),
              "rska_mrhs_tune")
        return int(c.value), float(u.value)

    def query(self, what: str) -> int:
        v = ctypes.c_int64()
        check(lib().rska_mrhs_query(self._h, MRHS_QUERY[what], ctypes.byref(v)), "rska_mrhs_query")
        return int(v.value)


class Unrolled:
    """K unrolled RSKA iterations on P problems with a hand-written adjoint
    (rska_unrolled_*).  Layout as for BatchSolver; call it with b (packed,
    float32 CUDA), lam and t (float32 CUDA tensors of P entries) to get the
    packed x_K as a differentiable function of (b, lam, t)."""

    def __init__(self, A: torch.Tensor, a_off, m, n, lda, b_off, eta: int, seed: int, K: int,
                 ckpt_every: int, stream=None):
        import numpy as np
        self.A = A
        self.P = len(m)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = A.device
        self._host = [np.ascontiguousarray(v, dtype=np.int64) for v in (a_off, m, n, lda, b_off)]
        ptrs = [ctypes.c_void_p(v.ctypes.data) for v in self._host]
        h = ctypes.c_void_p()
        check(lib().rska_unrolled_setup(ctypes.byref(h), self.P, _dptr(A), *ptrs, int(eta),
                                        int(seed), int(K), int(ckpt_every),
                                        _stream_ptr(self.stream)), "rska_unrolled_setup")
        self._h = h
        self.generation = 0
        self.x_off = np.zeros(self.P + 1, dtype=np.int64)
        check(lib().rska_unrolled_offsets(self._h, ctypes.c_void_p(self.x_off.ctypes.data)),
              "rska_unrolled_offsets")

    def close(self):
        if getattr(self, "_h", None):
            lib().rska_unrolled_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward_raw(self, b, lam, t):
        x = torch.empty(int(self.x_off[-1]), dtype=torch.float32, device=self.device)
        check(lib().rska_unrolled_forward(self._h, _dptr(b), _dptr(lam), _dptr(t), _dptr(x)),
              "rska_unrolled_forward")
        self._keep = (b, lam, t)
        self.generation += 1
        return x

    def backward_raw(self, gx, generation=None):
        # the library differentiates its most recent forward (its checkpoints
        # and the b, lambda, t it borrowed); a backward of an older forward
        # would silently differentiate at the wrong point
        if generation is not None and generation != self.generation:
            raise RuntimeError(
                f"rska_unrolled_backward: this output comes from forward {generation}, but "
                f"forward {self.generation} ran since; the adjoint only differentiates the most "
                "recent forward of an Unrolled context (run backward before the next forward)")
        b = self._keep[0]
        gb = torch.empty_like(b)
        glam = torch.empty(self.P, dtype=torch.float32, device=self.device)
        gt = torch.empty(self.P, dtype=torch.float32, device=self.device)
        check(lib().rska_unrolled_backward(self._h, _dptr(gx.contiguous()), _dptr(gb),
                                           _dptr(glam), _dptr(gt)), "rska_unrolled_backward")
        return gb, glam, gt

    def __call__(self, b, lam, t):
        return RSKAUnrolled.apply(b, lam, t, self)


class RSKAUnrolled(torch.autograd.Function):
    """x_K(b, lambda, t) of K unrolled RSKA iterations; the backward is the
    library's adjoint kernel (no autograd tape over the iterations)."""

    @staticmethod
    def forward(ctx, b, lam, t, unrolled):
        ctx.unrolled = unrolled
        x = unrolled.forward_raw(b.detach().contiguous(), lam.detach().contiguous(),
                                 t.detach().contiguous())
        ctx.generation = unrolled.generation
        return x

    @staticmethod
    def backward(ctx, gx):
        gb, glam, gt = ctx.unrolled.backward_raw(gx, ctx.generation)
        return gb, glam, gt, None
