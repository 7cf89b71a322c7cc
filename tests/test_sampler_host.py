"""The device sampler (csrc/rska_device.cuh: Philox4x32-10 and the alias draw
of the index contract, Algorithm 1's tau_k) compiled for the host and compared
word for word and index for index with the oracle's, over seeds, problem ids,
odd and even eta and iteration ranges.  CPU only; the GPU tests compare the
indices the kernels draw."""
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
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    so = str(tmp_path_factory.mktemp("sampler") / "libsampler_host.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", inc,
                    os.path.join(HERE, "host", "sampler_host.cpp"), "-o", so], check=True,
                   capture_output=True)
    L = ctypes.CDLL(so)
    L.host_sample.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_void_p]
    L.host_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return L


def test_philox_blocks_equal_the_oracle(orc, lib):
    rng = np.random.default_rng(11)
    for _ in range(200):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        out = np.zeros(4, np.uint32)
        lib.host_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data)
        np.testing.assert_array_equal(out, orc.philox4x32_10(ctr, key))


@pytest.mark.parametrize("m,eta,seed,problem,k0,K", [
    (1, 1, 0, 0, 0, 50),
    (7, 3, 5, 0, 0, 200),
    (1000, 10, 0, 0, 0, 100),
    (20000, 1024, 2**40 + 3, 0, 123456, 3),
    (333, 33, 0xFFFFFFFF, 4095, 2**33, 20),
    (4000, 32, 2024, 17, 7, 40),
])
def test_draws_equal_the_oracle(orc, lib, m, eta, seed, problem, k0, K):
    nu = np.random.default_rng(m + eta).chisquare(20, m) + 1e-3
    thr, alias = orc.alias_build(nu)
    out = np.zeros((K, eta), np.int32)
    lib.host_sample(thr.ctypes.data, alias.ctypes.data, m, seed, problem, k0, K, eta,
                    out.ctypes.data)
    np.testing.assert_array_equal(out, orc.sample(thr, alias, seed=seed, eta=eta, k0=k0, K=K,
                                                  problem=problem))
