"""ctypes loader for librska.so.  Fails loudly if the library is missing: there
is no CPU fallback for any entry point."""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librska.so")
_lib = None


class RSKAError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _load().rska_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")


def _declare(lib):
    P = ctypes.c_void_p
    i64, i32, u64, f32, f64, c_int = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_float, ctypes.c_double, ctypes.c_int)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "rska_setup": ([PP, P, i64, i64, i64, P, f32, i32, f32, u64, P], c_int),
        "rska_setup_host": ([PP, P, i64, i64, i64, P, f32, i32, f32, u64, P], c_int),
        "rska_load_host": ([P, P, P], c_int),
        "rska_solve": ([P, i64], c_int),
        "rska_solve_until": ([P, i64, i64, f64, P, ctypes.POINTER(i64), ctypes.POINTER(f64)],
                             c_int),
        "rska_get_x": ([P, P, P], c_int),
        "rska_set_state": ([P, P, i64], c_int),
        "rska_iteration": ([P, ctypes.POINTER(i64)], c_int),
        "rska_get_indices": ([P, i64, i64, P], c_int),
        "rska_get_tables": ([P, P, P, P], c_int),
        "rska_metrics": ([P, P, ctypes.POINTER(f64), ctypes.POINTER(f64)], c_int),
        "rska_reset": ([P], c_int),
        "rska_destroy": ([P], c_int),
        "rska_query": ([P, c_int, ctypes.POINTER(i64)], c_int),
        "rska_set_option": ([P, c_int, i64], c_int),
        "rska_set_weights": ([P, P, c_int], c_int),
        "rska_linearized_bregman": ([P, i64, f64], c_int),
        "rska_sigma_max2": ([P, i32, u64, ctypes.POINTER(f64), ctypes.POINTER(f64),
                             ctypes.POINTER(f64)], c_int),
        "rska_batch_setup": ([PP, i32, P, P, P, P, P, P, P, f32, i32, f32, u64, P], c_int),
        "rska_batch_set_stream_ids": ([P, P], c_int),
        "rska_batch_solve": ([P, i64, f64, i64], c_int),
        "rska_batch_results": ([P, P, P], c_int),
        "rska_batch_offsets": ([P, P], c_int),
        "rska_batch_get_x": ([P, P, P], c_int),
        "rska_batch_get_tables": ([P, P, P, P], c_int),
        "rska_batch_destroy": ([P], c_int),
        "rska_unrolled_setup": ([PP, i32, P, P, P, P, P, P, i32, u64, i32, i32, P], c_int),
        "rska_unrolled_forward": ([P, P, P, P, P], c_int),
        "rska_unrolled_backward": ([P, P, P, P, P], c_int),
        "rska_unrolled_offsets": ([P, P], c_int),
        "rska_unrolled_destroy": ([P], c_int),
        "rska_mrhs_setup": ([PP, P, i64, i64, i64, P, i64, i64, f32, i32, f32, u64, P], c_int),
        "rska_mrhs_set_option": ([P, c_int, i64], c_int),
        "rska_mrhs_query": ([P, c_int, ctypes.POINTER(i64)], c_int),
        "rska_mrhs_solve": ([P, i64], c_int),
        "rska_mrhs_tune": ([P, i32, ctypes.POINTER(i32), ctypes.POINTER(f64)], c_int),
        "rska_tune_candidates": ([i64, i64, i32, i32, P, i32, ctypes.POINTER(i32)], c_int),
        "rska_tune_cache": ([i32, ctypes.c_char_p, ctypes.POINTER(i32), ctypes.POINTER(f64)], c_int),
        "rska_mrhs_get_x": ([P, P, P], c_int),
        "rska_mrhs_get_indices": ([P, i64, i64, P], c_int),
        "rska_mrhs_get_tables": ([P, P, P, P], c_int),
        "rska_mrhs_reset": ([P], c_int),
        "rska_mrhs_destroy": ([P], c_int),
        "rska_solve_noalloc": ([P, i64, i64, i64, P, f32, i32, f32, u64, i64, P, P, P], c_int),
        "rska_probe_l2_read": ([P, i64, i32, i32, P, P], c_int),
        "rska_strerror": ([c_int], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"librska.so not found at {LIB_PATH}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def lib():
    return _load()


def check(code: int, where: str):
    if code != 0:
        raise RSKAError(code, where)
