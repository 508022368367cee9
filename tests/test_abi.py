"""Host-side checks of the C-ABI library: it builds, loads without a GPU, exports
every entry point the header declares, and validates plan arguments on the host
(no CUDA call is made by anything tested here)."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import paper_1807_07382_gb300 as pb
from paper_1807_07382_gb300 import _lib, build

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "pentbatch.h"


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z_0-9]*\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for required in ("pent_factor_batch", "pent_solve_batch", "pent_adjoint_solve_batch", "adi_step_2d"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_version_and_status_strings(L):
    assert L.pent_version().decode() == pb.__version__
    assert L.pent_status_string(_lib.PENT_ESINGULAR).decode() == "zero or non-finite pivot"


def _create(L, batch, n=None, n_uniform=0, shared=0, prec=0):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * len(n))(*n) if n is not None else None
    st = L.pent_plan_create(ctypes.byref(h), batch, arr, n_uniform, shared, prec, None)
    return st, h


@pytest.mark.parametrize("args", [
    dict(batch=0, n_uniform=8),
    dict(batch=4, n_uniform=0),
    dict(batch=3, n=[4, 0, 5]),
    dict(batch=2, n=[4, 5], shared=1),
    dict(batch=2, n_uniform=8, prec=7),
    dict(batch=2, n_uniform=40000, prec=1),     # FP32 refinement: n <= 32768 (a cluster of 8 CTAs)
])
def test_plan_create_rejects_bad_arguments(L, args):
    st, h = _create(L, **args)
    assert st == _lib.PENT_EINVAL
    assert not h.value


def test_plan_workspace_and_options(L):
    st, h = _create(L, batch=70, n_uniform=1024)
    assert st == 0
    ws = L.pent_plan_workspace_bytes(h)
    # FP64 records (5 doubles) + scratch (1 double) per padded row, 3 groups of 32
    assert ws >= 3 * 32 * 1024 * 6 * 8
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_BLOCK_WARPS, ctypes.byref(v)) == 0 and v.value >= 1
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_BLOCK_WARPS, 0) == _lib.PENT_EINVAL
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_BLOCK_WARPS, 2) == 0
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_THREADS_PER_SYSTEM, 32) == _lib.PENT_EINVAL
    assert L.pent_plan_set_option(h, 999, 1) == _lib.PENT_EINVAL
    # unbound plans refuse to work, without touching the GPU
    assert L.pent_solve_batch(h, ctypes.c_void_p(16), ctypes.c_void_p(16), 0) == _lib.PENT_ENOTBOUND
    assert L.pent_factor_hyperdiff(h, None) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)


def test_uneven_plan_workspace_counts_padded_groups(L):
    n = [64] * 31 + [1000]  # one group of 32: padded to the longest system
    st, h = _create(L, batch=32, n=n)
    assert st == 0
    assert L.pent_plan_workspace_bytes(h) >= 32 * 1000 * 6 * 8
    L.pent_plan_destroy(h)


def test_f32_threads_per_system_option_relayouts_before_bind(L):
    st, h = _create(L, batch=8, n_uniform=1024, prec=1)
    assert st == 0
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_THREADS_PER_SYSTEM, ctypes.byref(v)) == 0
    default_tps = v.value
    assert default_tps == 128
    base = L.pent_plan_workspace_bytes(h)
    for tps in (128, 256, 512, 1024, 2048):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_THREADS_PER_SYSTEM, tps) == 0
        # FP32 factors are 8 B per padded row (1/alpha and beta)
        assert L.pent_plan_workspace_bytes(h) >= 8 * 1024 * 8
    for bad in (48, 16, 32, 64, 1536 + 32, 8192):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_THREADS_PER_SYSTEM, bad) == _lib.PENT_EINVAL
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_THREADS_PER_SYSTEM, 0) == 0  # back to the automatic shape
    assert L.pent_plan_workspace_bytes(h) == base
    L.pent_plan_destroy(h)


def test_periodic_option_host_checks(L):
    # FP64, uniform n >= 5 only; before binding
    st, h = _create(L, batch=4, n_uniform=4)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 1) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    # FP32+refine periodic plans keep four FP32 planes per row (1/alpha, beta and the two columns of Z)
    st, h = _create(L, batch=4, n_uniform=64, prec=1)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 1) == 0
    assert L.pent_plan_workspace_bytes(h) >= 4 * 64 * 4 * 4  # systems x rows x planes x 4 B
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=2, n=[64, 65])
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 1) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=70, n_uniform=64)
    base = L.pent_plan_workspace_bytes(h)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 2) == _lib.PENT_EINVAL
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 1) == 0
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_PERIODIC, ctypes.byref(v)) == 0 and v.value == 1
    # nine interleaved planes of the reduced matrix (62 rows) per system, S^{-1}, and the g scratch
    assert L.pent_plan_workspace_bytes(h) >= (9 * 62 * 70 + 4 * 70 + 62 * 70) * 8
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 0) == 0
    assert L.pent_plan_workspace_bytes(h) == base
    L.pent_plan_destroy(h)


def test_new_entry_points_check_arguments_on_the_host(L):
    st, h = _create(L, batch=4, n_uniform=32)
    assert L.pent_step_batch(h, None, None, ctypes.c_void_p(16), 1, 0) == _lib.PENT_ENOTBOUND
    assert L.pent_refactor_solve_hyperdiff(h, None, ctypes.c_void_p(16), ctypes.c_void_p(16)) == _lib.PENT_EINVAL
    assert L.pent_refactor_solve_hyperdiff(h, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                           ctypes.c_void_p(16)) == _lib.PENT_ENOTBOUND
    L.pent_plan_destroy(h)


def test_cluster_warps_option_shapes(L):
    # FP32+refine only, 4 / 8 / 16, before binding; long systems become clusters of whole cw-warp CTAs
    st, h = _create(L, batch=3, n=[5000, 1000, 30000], prec=1)
    assert st == 0
    a, b = ctypes.c_int64(), ctypes.c_int64()
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_CLUSTER_WARPS, ctypes.byref(v)) == 0 and v.value == 8
    assert L.pent_plan_system_config(h, 0, ctypes.byref(a), ctypes.byref(b)) == 0
    assert (a.value, b.value) == (8, 768)  # 625 threads: three CTAs of 8 warps
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_CLUSTER_WARPS, 16) == 0
    assert L.pent_plan_system_config(h, 0, ctypes.byref(a), ctypes.byref(b)) == 0
    assert (a.value, b.value) == (8, 640)  # two CTAs of 10 warps under the 16-warp rule
    for cw, tps0 in ((8, 768), (4, 640)):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_CLUSTER_WARPS, cw) == 0
        assert L.pent_plan_system_config(h, 0, ctypes.byref(a), ctypes.byref(b)) == 0
        assert (a.value, b.value) == (8, tps0)  # ceil(625 / (32 cw)) CTAs of cw warps
        assert L.pent_plan_system_config(h, 1, ctypes.byref(a), ctypes.byref(b)) == 0
        assert b.value == 128  # 125 threads: one CTA of 4 warps
        assert L.pent_plan_system_config(h, 2, ctypes.byref(a), ctypes.byref(b)) == 0
        assert a.value * b.value >= 30000  # beyond 8 CTAs of cw warps: the 16-warp rule
    for bad in (0, 2, 12, 32):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_CLUSTER_WARPS, bad) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=2, n_uniform=64)  # FP64
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_CLUSTER_WARPS, 8) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)


def test_f32_refine_length_limit(L):
    # FP32+refine systems are at most a cluster of 8 CTAs x 512 threads x 8 rows; FP64 takes any length
    for n, want32 in ((32768, 0), (32769, _lib.PENT_EINVAL), (100000, _lib.PENT_EINVAL)):
        st, h = _create(L, batch=1, n=[n], prec=1)
        assert st == want32
        if st == 0:
            L.pent_plan_destroy(h)
        st, h = _create(L, batch=1, n=[n])
        assert st == 0
        L.pent_plan_destroy(h)


def test_fp32_kernel_option(L):
    """PENT_OPT_FP32_KERNEL: 0 (interior-constant kernel where it applies) or 1 (general
    kernel), FP32 plans only; settable at any time, readable back."""
    st, h = _create(L, batch=4, n_uniform=64, prec=1)
    assert st == 0
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_FP32_KERNEL, ctypes.byref(v)) == 0 and v.value == 0
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_FP32_KERNEL, 2) == _lib.PENT_EINVAL
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_FP32_KERNEL, 1) == 0
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_FP32_KERNEL, ctypes.byref(v)) == 0 and v.value == 1
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=4, n_uniform=64, prec=0)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_FP32_KERNEL, 1) == _lib.PENT_EINVAL  # FP64 plan
    L.pent_plan_destroy(h)


def test_adi_plans_factor_and_graph_cache_query_check_arguments_on_the_host(L):
    st, px = _create(L, batch=8, n_uniform=16, shared=1)
    st2, py = _create(L, batch=16, n_uniform=8, shared=1)
    assert st == 0 and st2 == 0
    assert L.adi_plans_factor(None, py, 0.01, 1e-6, 1 / 16) == _lib.PENT_EINVAL
    assert L.adi_plans_factor(px, px, 0.01, 1e-6, 1 / 16) == _lib.PENT_EINVAL
    assert L.adi_plans_factor(px, py, -0.01, 1e-6, 1 / 16) == _lib.PENT_EINVAL
    assert L.adi_plans_factor(px, py, 0.01, 0.0, 1 / 16) == _lib.PENT_EINVAL
    assert L.adi_plans_factor(px, py, 0.01, 1e-6, 1 / 16) == _lib.PENT_ENOTBOUND  # nothing launched
    v = ctypes.c_int64(-1)
    assert L.pent_plan_get_option(px, _lib.PENT_OPT_CACHED_GRAPHS, ctypes.byref(v)) == 0 and v.value == 0
    assert L.pent_plan_set_option(px, _lib.PENT_OPT_CACHED_GRAPHS, 3) == _lib.PENT_EINVAL  # read only
    L.pent_plan_destroy(px)
    L.pent_plan_destroy(py)


@pytest.mark.parametrize("R", [1024, 2048, 4096])
def test_window_layout_tiles_every_length(L, R):
    """pent_window_layout: the kept rows of the windows tile [0, n) once, every window has at
    most R rows and lies inside the system, each cut is at least the overlap away from the
    rows a window keeps, and windows start on multiples of 8 rows."""
    for O in (8, 16, 96, R // 8, R // 4):
        for n in list(range(R + 1, R + 40)) + [2 * R - 2 * O, 2 * R - 2 * O + 1, 3 * R, 5 * R + 7, 16384, 65536 + 3]:
            w = pb.window_layout(n, R, O)
            assert len(w) >= 2
            kept = np.concatenate([np.arange(a + k0, a + k1) for a, m, k0, k1 in w])
            assert np.array_equal(kept, np.arange(n))
            for i, (a, m, k0, k1) in enumerate(w):
                assert a % 8 == 0 and 0 < m <= R and a + m <= n
                assert (a == 0) == (i == 0) and (a + m == n) == (i == len(w) - 1)
                assert k0 == (0 if a == 0 else O) and k1 == (m if a + m == n else m - O)
                assert k1 > k0
            # the count never falls as the overlap grows (the workspace is sized for the largest)
            if O < R // 4:
                assert len(w) <= len(pb.window_layout(n, R, R // 4))
    for n, R2, O in ((R, R, 8), (100, R, 8), (5 * R, R, 0), (5 * R, R, 12), (5 * R, R, R // 4 + 8), (5 * R, 1004, 8)):
        assert len(pb.window_layout(n, R2, O)) == 0


def test_window_warps_option_host_checks(L):
    """PENT_OPT_WINDOW_WARPS: FP32+refine, non-periodic, before binding, 0 / 4 / 8 / 16; it
    resizes the workspace by the windows' overlap room.  PENT_OPT_WINDOWS is read only (0
    before any factorisation)."""
    st, h = _create(L, batch=3, n=[16384, 1000, 5000], prec=1)
    assert st == 0
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_WINDOW_WARPS, ctypes.byref(v)) == 0 and v.value == 4
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_WINDOWS, ctypes.byref(v)) == 0 and v.value == 0
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOWS, 1) == _lib.PENT_EINVAL
    sizes = {}
    for w in (0, 4, 8, 16):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_WARPS, w) == 0
        sizes[w] = L.pent_plan_workspace_bytes(h)
    # the reserve: per window 2 (R / 8) doubles of overlap rows and one int4, per system an int32
    for w in (4, 8, 16):
        R = 256 * w
        nwin = sum(len(pb.window_layout(n, R, R // 8)) for n in (16384, 1000, 5000))
        assert sizes[w] - sizes[0] >= nwin * 2 * (R // 8) * 8 - 3 * 256  # 256-byte aligned regions
        assert sizes[w] - sizes[0] <= nwin * (2 * (R // 8) * 8 + 16) + 3 * 4 + 4096
    for bad in (1, 2, 12, 32, -1):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_WARPS, bad) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=2, n_uniform=8192)  # FP64
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_WARPS, 4) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=2, n_uniform=8192, prec=1)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 1) == 0
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_WARPS, 4) == _lib.PENT_EINVAL  # periodic
    L.pent_plan_destroy(h)


def test_window_rows_option_host_checks(L):
    """PENT_OPT_WINDOW_ROWS: FP64 per-system plans, before binding, 0 or a multiple of 64 in
    256 .. 16384 (default 1024); the workspace grows by the windows' side scratch and overlap
    rows (three times omax / 2 row pairs of 32 lanes a window) when a group is longer than one window."""
    st, h = _create(L, batch=64, n=[5000] * 32 + [300] * 32)
    assert st == 0
    v = ctypes.c_int64()
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_WINDOW_ROWS, ctypes.byref(v)) == 0 and v.value == 1024
    base = L.pent_plan_workspace_bytes(h)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_ROWS, 0) == 0
    off = L.pent_plan_workspace_bytes(h)
    nwin = len(pb.window_layout(5000, 1024, 128))
    assert base - off >= nwin * 3 * 64 * 32 * 16 - 4 * 256
    for bad in (100, 255, 1000, 16448, -4):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_ROWS, bad) == _lib.PENT_EINVAL
    for good in (256, 512, 2048, 16384):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_ROWS, good) == 0
    L.pent_plan_destroy(h)
    for kw in (dict(n_uniform=5000, shared=1), dict(n_uniform=5000, prec=1)):  # shared; FP32
        st, h = _create(L, batch=8, **kw)
        assert st == 0
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_ROWS, 1024) == _lib.PENT_EINVAL
        L.pent_plan_destroy(h)


def test_persistent_option_host_checks(L):
    """PENT_OPT_PERSISTENT: 0 or 1, any precision but periodic plans, at any time; readable back."""
    for prec in (0, 1):
        st, h = _create(L, batch=4, n_uniform=5000, prec=prec)
        assert st == 0
        v = ctypes.c_int64(-1)
        assert L.pent_plan_get_option(h, _lib.PENT_OPT_PERSISTENT, ctypes.byref(v)) == 0 and v.value == 0
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERSISTENT, 2) == _lib.PENT_EINVAL
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERSISTENT, 1) == 0
        assert L.pent_plan_get_option(h, _lib.PENT_OPT_PERSISTENT, ctypes.byref(v)) == 0 and v.value == 1
        L.pent_plan_destroy(h)
    st, h = _create(L, batch=4, n_uniform=64)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERIODIC, 1) == 0
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_PERSISTENT, 1) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)


def test_fp64_interior_option_host_checks(L):
    """PENT_OPT_FP64_INTERIOR: FP64 plans only, 0 or 1 (default 1), at any time."""
    st, h = _create(L, batch=4, n_uniform=1024)
    v = ctypes.c_int64(-1)
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_FP64_INTERIOR, ctypes.byref(v)) == 0 and v.value == 1
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_FP64_INTERIOR, 0) == 0
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_FP64_INTERIOR, ctypes.byref(v)) == 0 and v.value == 0
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_FP64_INTERIOR, 2) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=4, n_uniform=1024, prec=1)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_FP64_INTERIOR, 1) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)


def test_window_form_option_host_checks(L):
    """PENT_OPT_WINDOW_FORM: FP64 plans, before binding, 0 (group windows) or 1 (system windows,
    the default); system windows reserve a per-system copy of the windowed systems' records
    (80 bytes a row pair) in place of the group windows' side scratch and overlap rows."""
    st, h = _create(L, batch=64, n=[5000] * 32 + [300] * 32)
    assert st == 0
    v = ctypes.c_int64(-1)
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_WINDOW_FORM, ctypes.byref(v)) == 0 and v.value == 1
    ws1 = L.pent_plan_workspace_bytes(h)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_FORM, 0) == 0
    assert L.pent_plan_get_option(h, _lib.PENT_OPT_WINDOW_FORM, ctypes.byref(v)) == 0 and v.value == 0
    ws0 = L.pent_plan_workspace_bytes(h)
    group_room = len(pb.window_layout(5000, 1024, 128)) * 64 * 32 * 48  # side + halo of the group windows
    assert ws1 - ws0 >= 32 * 2500 * 80 - group_room
    for bad in (2, -1):
        assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_FORM, bad) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)
    st, h = _create(L, batch=8, n_uniform=5000, prec=1)
    assert L.pent_plan_set_option(h, _lib.PENT_OPT_WINDOW_FORM, 0) == _lib.PENT_EINVAL
    L.pent_plan_destroy(h)


@pytest.mark.parametrize("R", [256, 1024, 2048])
def test_system_window_layout_tiles_every_length(L, R):
    """pent_system_window_layout (FP64 system windows): the kept rows tile [0, n) once, every
    window of a system walks the same min(R, n rounded up to a pair) rows starting at an even row,
    and every kept row is at least O from each cut (a cut is a window edge inside the system)."""
    for O in (8, 16, R // 8, R // 4):
        for n in list(range(1, 3 * R + 3, 7)) + [R - 1, R, R + 1, R + 2, 2 * R - 2 * O, 2 * R - 2 * O + 1, 40001]:
            w = pb.system_window_layout(n, R, O)
            assert len(w) >= 1
            walk = min(R, 2 * ((n + 1) // 2))
            cur = 0
            for r0, k0, k1 in w:
                assert r0 % 2 == 0 and r0 <= k0 < k1 <= n and k0 == cur
                assert r0 + walk <= 2 * ((n + 1) // 2)
                assert r0 == 0 or k0 - r0 >= O
                assert r0 + walk >= n or r0 + walk - k1 >= O
                cur = k1
            assert cur == n
            if n <= R:
                assert w.tolist() == [[0, 0, n]]
    assert len(pb.system_window_layout(3000, R, R // 4 + 2)) == 0  # more overlap than a quarter window
    assert len(pb.system_window_layout(3000, R, 7)) == 0             # odd overlap
    assert len(pb.system_window_layout(0, R, 8)) == 0
