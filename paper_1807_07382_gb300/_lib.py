"""ctypes declarations of the C ABI in include/pentbatch.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import threading
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libpentbatch.so"

# status codes
PENT_OK = 0
PENT_EINVAL = -1
PENT_ESINGULAR = -2
PENT_ENOCONV = -3
PENT_ECUDA = -4
PENT_ENOTFACTORED = -5
PENT_ENOTBOUND = -6

PENT_F64 = 0
PENT_F32_REFINE = 1

PENT_RESIDUAL_FF = 0
PENT_RESIDUAL_F64 = 1

PENT_OPT_THREADS_PER_SYSTEM = 1
PENT_OPT_RESIDUAL = 2
PENT_OPT_BLOCK_WARPS = 3
PENT_OPT_REFINE_TOL_LOG2 = 4
PENT_OPT_UNROLL = 5
PENT_OPT_ROWS_PER_THREAD = 6
PENT_OPT_PARTITION_ROWS = 7
PENT_OPT_PERIODIC = 8
PENT_OPT_CLUSTER_WARPS = 9
PENT_OPT_FP32_KERNEL = 10
PENT_OPT_CACHED_GRAPHS = 11
PENT_OPT_WINDOW_WARPS = 12
PENT_OPT_WINDOWS = 13
PENT_OPT_WINDOW_ROWS = 14
PENT_OPT_PERSISTENT = 15
PENT_OPT_FP64_INTERIOR = 16
PENT_OPT_WINDOW_FORM = 17
PENT_MAX_CACHED_GRAPHS = 16

# every symbol the header declares, with (restype, argtypes)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)

SIGNATURES = {
    "pent_plan_create": (_int, [ctypes.POINTER(_vp), _i64, _i64p, _i64, _int, _int, ctypes.c_char_p]),
    "pent_plan_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "pent_plan_bind": (_int, [_vp, _vp, _vp]),
    "pent_plan_set_option": (_int, [_vp, _int, _i64]),
    "pent_plan_get_option": (_int, [_vp, _int, _i64p]),
    "pent_plan_system_config": (_int, [_vp, _i64, _i64p, _i64p]),
    "pent_factor_batch": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "pent_factor_hyperdiff": (_int, [_vp, _vp]),
    "pent_solve_batch": (_int, [_vp, _vp, _vp, _int]),
    "pent_solve_steps": (_int, [_vp, _vp, _i64, _int]),
    "pent_solve_host_batch": (_int, [_vp, _vp, _vp, _vp, _vp, _int, _int]),
    "pent_host_range_mapped": (_int, [_vp, ctypes.c_size_t]),
    "pent_step_batch": (_int, [_vp, _vp, _vp, _vp, _i64, _int]),
    "pent_refactor_solve_hyperdiff": (_int, [_vp, _vp, _vp, _vp]),
    "pent_adjoint_solve_batch": (_int, [_vp, _vp, _vp, _int]),
    "pent_hyperdiff_sigma_grad": (_int, [_vp, _vp, _vp, _vp]),
    "adi_step_2d": (_int, [_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _dbl, _int]),
    "adi_plans_factor": (_int, [_vp, _vp, _dbl, _dbl, _dbl]),
    "adi_steps_2d": (_int, [_vp, _vp, _vp, _i64, _i64, _dbl, _dbl, _dbl, _int, _i64]),
    "pent_get_info": (_int, [_vp, _i64p, _i64p, _intp]),
    "pent_clear_info": (_int, [_vp]),
    "pent_gbsv_batch_noalloc": (_int, [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pent_probe_fp64_fma": (_int, [_i64, _i64, _vp, _vp, ctypes.POINTER(_dbl)]),
    "pent_window_layout": (_i64, [_i64, _int, _int, _vp, _i64]),
    "pent_system_window_layout": (_i64, [_i64, _int, _int, _vp, _i64]),
    "pent_plan_destroy": (None, [_vp]),
    "pent_status_string": (ctypes.c_char_p, [_int]),
    "pent_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class PentError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _status_text(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def _status_text(status: int) -> str:
    try:
        return load().pent_status_string(status).decode()
    except Exception:  # noqa: BLE001 - best effort text only
        return "status"


def load(path: Path | None = None):
    """Load libpentbatch.so (built by build.py).  Raises if it is missing: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            p = Path(path) if path else LIB_PATH
            if not p.exists():
                raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_1807_07382_gb300/build.py)")
            L = ctypes.CDLL(str(p))
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str = "") -> None:
    if status != PENT_OK:
        raise PentError(status, what)
