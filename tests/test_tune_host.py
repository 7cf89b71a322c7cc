"""The multi-right-hand-side autotuner's host logic (no device work): the
candidate schedules it times and the cache of its choices, through the C ABI
(rska_tune_candidates, rska_tune_cache).  CPU only."""
import os

import pytest


@pytest.fixture(scope="module")
def rska():
    from paper_2203_10838_gb300 import build
    build.build()
    from paper_2203_10838_gb300 import rska as r
    return r


def test_candidates_of_the_benchmark_configuration(rska):
    # 16384 x 8192, 512 right-hand sides, eta = 256 on 152 SMs: the staged form
    # with four splits x programmatic launch on/off, and the persistent form
    # (32 column slices x 4 right-hand-side slices = 128 CTAs) with six
    # gather schedules
    codes = rska.tune_candidates(8192, 512, 256, 152)
    assert len(codes) == len(set(codes)) == 14
    dec = [rska.decode_schedule(c) for c in codes]
    staged = {(d["ksplit"], d["pdl"]) for d in dec if d["form"] == "staged"}
    assert staged == {(k, p) for k in (0, 16, 32, 64) for p in (0, 1)}
    # with the residual product, after the barrier, after each of the
    # scaled residual's four 64-row chunks
    assert {d["gather_sched"] for d in dec if d["form"] == "persistent"} == {0, 1, 2, 3, 4, 5}


def test_candidates_respect_each_form_s_limits(rska):
    # eta above 256: no persistent candidate
    assert all(rska.decode_schedule(c)["form"] == "staged"
               for c in rska.tune_candidates(8192, 512, 300, 152))
    # too many CTAs for the persistent form (64 x 4 > 152 SMs)
    assert all(rska.decode_schedule(c)["form"] == "staged"
               for c in rska.tune_candidates(16384, 512, 256, 152))
    # n = 300 (8 blocks of 64 columns): splits above 8 are left out
    dec = [rska.decode_schedule(c) for c in rska.tune_candidates(300, 40, 100, 152)]
    assert {d.get("ksplit") for d in dec if d["form"] == "staged"} == {0}
    # eta = 100 pads to two 64-row chunks: gather schedules 0, 1, 2 and 3
    assert sorted(d["gather_sched"] for d in dec if d["form"] == "persistent") == [0, 1, 2, 3]
    # every candidate fits in the table that rska_mrhs_tune uses
    for n, R, eta in [(8192, 512, 256), (1, 1, 1), (100000, 4096, 4096)]:
        assert 1 <= len(rska.tune_candidates(n, R, eta, 152)) <= 32


def test_cache_round_trip(rska, tmp_path):
    rska.tune_cache("clear")
    assert rska.tune_cache("get", "mrhs:test:a") is None
    rska.tune_cache("put", "mrhs:test:a", 2 | (1 << 17), 6.25)
    rska.tune_cache("put", "mrhs:test:b", 1 | (32 << 8) | (1 << 16), 24.5)
    assert rska.tune_cache("get", "mrhs:test:a") == (2 | (1 << 17), 6.25)
    path = str(tmp_path / "tune.txt")
    rska.tune_cache("save", path)
    assert len(open(path).read().splitlines()) == 2
    rska.tune_cache("clear")
    assert rska.tune_cache("get", "mrhs:test:b") is None
    rska.tune_cache("load", path)
    assert rska.tune_cache("get", "mrhs:test:b") == (1 | (32 << 8) | (1 << 16), 24.5)
    from paper_2203_10838_gb300._lib import RSKAError
    with pytest.raises(RSKAError):
        rska.tune_cache("put", "a key with spaces", 1, 1.0)
    with pytest.raises(RSKAError):
        rska.tune_cache("load", os.path.join(str(tmp_path), "missing.txt"))
    rska.tune_cache("clear")
