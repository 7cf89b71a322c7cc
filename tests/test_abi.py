"""CPU checks of the C ABI: the library loads, exports every entry point that
include/rska.h declares, and rejects bad arguments on the host before any
CUDA call is made.  No kernel runs here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2203_10838_gb300 import build
    build.build()
    from paper_2203_10838_gb300._lib import lib
    return lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(rska\w*)\s*\(", src))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["rska_setup", "rska_solve", "rska_get_x", "rska_destroy", "rska_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(L):
    from paper_2203_10838_gb300._lib import LIB_PATH
    raw = ctypes.CDLL(LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(raw, n)]
    assert not missing, missing


def test_strerror_covers_codes(L):
    for code in range(0, 8):
        assert L.rska_strerror(code)
    assert L.rska_strerror(12345) == b"unknown error"


FAKE = ctypes.c_void_p(0x10000)   # 16-byte aligned, never dereferenced


@pytest.mark.parametrize("args", [
    dict(A=None),
    dict(b=None),
    dict(m=0),
    dict(n=0),
    dict(lda=10),            # lda < n
    dict(lda=18, n=16),      # lda not a multiple of 4
    dict(eta=0),
    dict(eta=4097),
    dict(lam=-1.0),
    dict(lam=float("nan")),
    dict(t=0.0),
    dict(t=float("inf")),
    dict(A=ctypes.c_void_p(0x10004)),   # misaligned A
])
def test_setup_rejects_bad_arguments_before_touching_the_device(L, args):
    p = dict(A=FAKE, b=FAKE, m=100, n=16, lda=16, lam=1.0, eta=8, t=1.0)
    p.update(args)
    h = ctypes.c_void_p(0xDEAD)
    rc = L.rska_setup(ctypes.byref(h), p["A"], p["m"], p["n"], p["lda"], p["b"], p["lam"],
                      p["eta"], p["t"], 0, None)
    assert rc == 1
    assert h.value is None


def test_null_context_is_rejected(L):
    assert L.rska_solve(None, 1) == 1
    assert L.rska_get_x(None, None, None) == 1
    assert L.rska_destroy(None) == 1
    assert L.rska_metrics(None, None, None, None) == 1
    k = ctypes.c_int64()
    assert L.rska_iteration(None, ctypes.byref(k)) == 1
    assert L.rska_set_weights(None, None, 0) == 1
    assert L.rska_set_weights(None, None, 2) == 1
    s2 = ctypes.c_double()
    assert L.rska_sigma_max2(None, 10, 0, ctypes.byref(s2), None, None) == 1
    assert L.rska_linearized_bregman(None, 1, 1.0) == 1
    h = ctypes.c_void_p()
    assert L.rska_setup_host(ctypes.byref(h), None, 10, 10, 12, None, 1.0, 4, 1.0, 0, None) == 1


@pytest.mark.parametrize("args", [
    dict(A=None),
    dict(B=None),
    dict(m=0),
    dict(n=0),
    dict(R=0),
    dict(lda=8, n=16),       # lda < n
    dict(lda=20, n=16),      # lda not a multiple of 8
    dict(ldb=50),            # ldb < m
    dict(eta=0),
    dict(eta=4097),
    dict(lam=-1.0),
    dict(t=0.0),
    dict(A=ctypes.c_void_p(0x10008)),   # A not 16-byte aligned
])
def test_mrhs_setup_rejects_bad_arguments_before_touching_the_device(L, args):
    p = dict(A=FAKE, B=FAKE, m=100, n=16, lda=16, R=4, ldb=100, lam=1.0, eta=8, t=1.0)
    p.update(args)
    h = ctypes.c_void_p(0xDEAD)
    rc = L.rska_mrhs_setup(ctypes.byref(h), p["A"], p["m"], p["n"], p["lda"], p["B"], p["R"],
                           p["ldb"], p["lam"], p["eta"], p["t"], 0, None)
    assert rc == 1
    assert h.value is None


def test_mrhs_null_context_is_rejected(L):
    assert L.rska_mrhs_solve(None, 1) == 1
    assert L.rska_mrhs_get_x(None, None, None) == 1
    assert L.rska_mrhs_set_option(None, 0, 2) == 1
    assert L.rska_mrhs_reset(None) == 1
    assert L.rska_mrhs_destroy(None) == 1
    v = ctypes.c_int64()
    assert L.rska_mrhs_query(None, 0, ctypes.byref(v)) == 1


@pytest.mark.parametrize("args", [
    dict(buf=None),                       # null buffer
    dict(sink=None),                      # null sink
    dict(nbytes=8),                       # fewer than 16 bytes
    dict(nbytes=1000),                    # not a multiple of 16
    dict(reps=0),
    dict(ctas=0),
    dict(buf=ctypes.c_void_p(0x10008)),   # not 16-byte aligned
])
def test_l2_probe_rejects_bad_arguments_before_launching(L, args):
    p = dict(buf=ctypes.c_void_p(0x10000), nbytes=1 << 20, reps=1, ctas=4,
             sink=ctypes.c_void_p(0x20000))
    p.update(args)
    assert L.rska_probe_l2_read(p["buf"], p["nbytes"], p["reps"], p["ctas"], p["sink"], None) == 1
