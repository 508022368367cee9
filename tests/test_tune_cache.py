"""Host-side checks of the autotuning cache: parsing, which rule each system
takes, precedence of options over the cache, and rejection of malformed
caches (pent_plan_create, pent_plan_system_config; no CUDA call)."""
import ctypes
import math

import pytest

from paper_1807_07382_gb300 import _lib, autotune, build

F64, F32 = _lib.PENT_F64, _lib.PENT_F32_REFINE


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def create(L, ns, prec, cache=None):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * len(ns))(*ns)
    st = L.pent_plan_create(ctypes.byref(h), len(ns), arr, 0, 0, prec, str(cache).encode() if cache else None)
    return st, h


def config(L, h, s):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    assert L.pent_plan_system_config(h, s, ctypes.byref(a), ctypes.byref(b)) == 0
    return a.value, b.value


def test_f32_rules_pick_each_systems_shape(L, tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("# comment line\n"
                     "f32 1 256 4 0      # fewest threads of 4 rows\n"
                     "f32 257 2048 8 512\n"
                     "f32 2049 100000 8 0\n"
                     "f64 1 100000 8 1\n")
    ns = [100, 256, 300, 2048, 5000, 30000]
    st, h = create(L, ns, F32, cache)
    assert st == 0
    try:
        assert config(L, h, 0) == (4, 32)        # ceil(100 / 4) = 25 threads -> one warp
        assert config(L, h, 1) == (4, 64)
        assert config(L, h, 2) == (8, 512)       # explicit threads per system
        assert config(L, h, 3) == (8, 512)
        assert config(L, h, 4) == (8, 768)       # 625 threads -> cluster of 3 CTAs x 8 warps
        assert config(L, h, 5) == (8, 3840)      # 3750 threads -> 8 CTAs x 15 warps
    finally:
        L.pent_plan_destroy(h)
    # 40,000 rows at 8 per thread need more than 8 CTAs of 16 warps: rejected
    st, _ = create(L, [40000], F32, cache)
    assert st == _lib.PENT_EINVAL


def test_f32_rule_that_cannot_hold_its_systems_is_rejected(L, tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("f32 1 5000 4 64\n")  # 64 threads x 4 rows = 256 < 5000
    st, _ = create(L, [100, 5000], F32, cache)
    assert st == _lib.PENT_EINVAL


@pytest.mark.parametrize("text", [
    "f16 1 10 4 0\n",            # unknown kind
    "f32 1 10 5 0\n",            # rows per thread must be 4 or 8
    "f32 1 10 4 48\n",           # threads per system not a multiple of 32
    "f32 10 1 4 0\n",            # n_hi < n_lo
    "f32 0 10 4 0\n",            # n_lo < 1
    "f64 1 10 3 2\n",            # unroll 2, 4 or 8
    "f64 1 10 4 9\n",            # warps per CTA 1..8
    "f64 1 10 4\n",              # missing field
    "f64 1 10 4 2 7\n",          # extra field
])
def test_malformed_cache_is_rejected(L, tmp_path, text):
    cache = tmp_path / "bad.txt"
    cache.write_text(text)
    for prec in (F64, F32):
        st, _ = create(L, [64, 128], prec, cache)
        assert st == _lib.PENT_EINVAL


def test_missing_cache_file_is_rejected(L, tmp_path):
    st, _ = create(L, [64], F64, tmp_path / "does_not_exist.txt")
    assert st == _lib.PENT_EINVAL


def test_f64_groups_take_the_rule_of_their_longest_system(L, tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("f64 1 1000 2 4\nf64 1001 20000 8 1\n")
    # 64 long systems (two groups of 32) and 40 short ones (groups sorted longest first)
    ns = [4000] * 64 + [500] * 40
    st, h = create(L, ns, F64, cache)
    assert st == 0
    try:
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_PARTITION_ROWS, 0) == 0  # every group walked whole
        for s in range(64):
            assert config(L, h, s) == (8, 1)
        for s in range(64, 104):
            assert config(L, h, s) == (2, 4)
        # an explicit option applies to every group
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_UNROLL, 4) == 0
        for s in (0, 70):
            assert config(L, h, s)[0] == 4
    finally:
        L.pent_plan_destroy(h)


def test_options_take_precedence_over_the_cache(L, tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("f32 1 100000 4 0\n")
    st, h = create(L, [1024, 1024], F32, cache)
    assert st == 0
    try:
        assert config(L, h, 0) == (4, 256)
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_ROWS_PER_THREAD, 8) == 0
        assert config(L, h, 0) == (8, 128)
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_THREADS_PER_SYSTEM, 256) == 0
        assert config(L, h, 1) == (8, 256)
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_ROWS_PER_THREAD, 5) == _lib.PENT_EINVAL
    finally:
        L.pent_plan_destroy(h)


def test_without_cache_the_built_in_choice_applies(L):
    st, h = create(L, [100, 1024, 3000], F32)
    assert st == 0
    try:
        assert config(L, h, 0) == (4, 32)
        assert config(L, h, 1) == (8, 128)
        assert config(L, h, 2) == (8, 384)
    finally:
        L.pent_plan_destroy(h)


def test_autotuner_candidates_cover_their_bucket():
    for n in autotune.DEFAULT_BUCKETS + (100, 3000, 20000, 32768):
        cands = autotune.f32_candidates(n)
        assert cands
        for rpt, tps in cands:
            assert rpt in (4, 8) and tps % 32 == 0 and rpt * tps >= n
            assert tps <= 512 or (tps % 512 == 0 and tps // 512 <= 8)


def test_cache_text_round_trips_through_the_parser(L, tmp_path):
    rules = [("f64", 1, 1024, 4, 2, 0.5), ("f32", 1, 1024, 8, 0, 0.4), ("f64", 1025, 16384, 8, 1, 9.0),
             ("f32", 1025, 16384, 8, 0, 2.0)]
    cache = tmp_path / "tune.txt"
    cache.write_text(autotune.format_cache(rules, header="test"))
    for prec in (F64, F32):
        st, h = create(L, [1000, 20000], prec, cache)
        assert st == 0
        if prec == F32:
            assert config(L, h, 1) == (8, 2560)   # 20000 / 8 = 2500 threads -> 5 CTAs of 16 warps
        else:
            assert config(L, h, 1) == (0, 256)    # 20,000 rows: partitioned automatically
            assert L.pent_plan_set_option(h, _lib.PENT_OPT_PARTITION_ROWS, 0) == 0
            assert config(L, h, 1) == (8, 1)      # the last rule extends to longer systems
        L.pent_plan_destroy(h)


def test_long_groups_are_partitioned_automatically(L):
    # 64 systems of 16,384 rows (two groups) and 1,000 of 100: 1.2 M rows, threshold 2,048 rows
    ns = [16384] * 64 + [100] * 1000
    st, h = create(L, ns, F64)
    assert st == 0
    try:
        assert config(L, h, 0) == (0, 256)           # partitioned, 256-row chunks
        assert config(L, h, 63) == (0, 256)
        assert config(L, h, 64)[0] in (2, 4, 8)      # short systems keep the thread-per-system walk
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_PARTITION_ROWS, 0) == 0
        assert config(L, h, 0)[0] in (2, 4, 8)
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_PARTITION_ROWS, 50) == 0
        assert config(L, h, 64) == (0, 256)
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_PARTITION_ROWS, -2) == _lib.PENT_EINVAL
    finally:
        L.pent_plan_destroy(h)
    # a uniform batch of 1024-row systems that fills the GPU (65,536 systems, 2,048 groups) keeps the
    # thread-per-system walk; a small one (4,096 systems, 128 groups) is cut into chunks from 512 rows
    st, h = create(L, [1024] * 65536, F64)
    assert st == 0 and config(L, h, 0)[0] in (2, 4, 8)
    L.pent_plan_destroy(h)
    st, h = create(L, [1024] * 4096, F64)
    assert st == 0 and config(L, h, 0) == (0, 256)
    L.pent_plan_destroy(h)
    st, h = create(L, [500] * 4096, F64)
    assert st == 0 and config(L, h, 0)[0] in (2, 4, 8)
    L.pent_plan_destroy(h)
