"""The device alias construction (csrc/rska_alias.cuh: the small/large test,
the pairing loop with the pushed entry kept in registers, the thresholds)
compiled for the host and compared bit for bit with the oracle's Vose table
(Sec. 5: p_i = ||a_i||^2 / ||A||_F^2), one thread and block partitions of 1 to
1024 threads, on 48 inputs: chi-square, uniform, exponential, one heavy row,
small integers and log-normal weights, m from 1 to 20000.  CPU only; the GPU
tests compare the tables the kernels build."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda_runtime.h")) else None


@pytest.fixture(scope="module")
def host_alias(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    so = str(tmp_path_factory.mktemp("alias") / "libalias_host.so")
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", "-I", inc,
                    os.path.join(HERE, "host", "alias_host.cpp"), "-o", so], check=True,
                   capture_output=True)
    L = ctypes.CDLL(so)
    L.host_alias.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_int]

    def run(nu, mode):
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        m = len(nu)
        thr = np.zeros(m, np.uint32)
        al = np.zeros(m, np.int32)
        L.host_alias(nu.ctypes.data, m, thr.ctypes.data, al.ctypes.data, mode)
        return thr, al
    return run


def _inputs():
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 5, 17, 100, 1000, 20000):
        heavy = np.ones(m)
        heavy[0] = 1e6
        yield rng.chisquare(50, m) + 0.0
        yield np.ones(m)
        yield rng.exponential(1.0, m) + 1e-9
        yield heavy
        yield rng.integers(1, 4, m).astype(np.float64)
        yield np.exp(rng.normal(0, 3, m))


def test_device_alias_tables_equal_the_oracle(orc, host_alias):
    n = 0
    for nu in _inputs():
        thr, alias = orc.alias_build(nu)
        for mode in (0, 1, 7, 256, 1024):   # 0: one thread; else block partitions
            t2, a2 = host_alias(nu, mode)
            np.testing.assert_array_equal(t2, thr, err_msg=f"m={len(nu)} mode={mode}")
            np.testing.assert_array_equal(a2, alias, err_msg=f"m={len(nu)} mode={mode}")
            n += 1
    assert n == 240
