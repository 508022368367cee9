"""Batched pentadiagonal factor-once / solve-many on one GB300 GPU.

Python binding of the C ABI in include/pentbatch.h.  Every step of the solve
runs in the library's CUDA kernels; this module only marshals arguments.
PyTorch supplies device memory (the plan's workspace and the caller's
vectors) and the CUDA stream.  There is no CPU fallback: if the CUDA library
is missing, or a tensor is not on a CUDA device, the calls raise.

Method: Gloster, O Naraigh and Pang, "cuPentBatch -- A batched pentadiagonal
solver for NVIDIA GPUs" (arXiv 1807.07382), Sec. 2.4 (LU without pivoting,
forward and back substitution) and Sec. 2.6 (factor once, solve many).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

from . import _lib
from ._lib import (PENT_ENOCONV, PENT_ESINGULAR, PENT_F32_REFINE, PENT_F64, PENT_OK, PENT_OPT_BLOCK_WARPS,
                   PENT_OPT_CLUSTER_WARPS, PENT_OPT_FP32_KERNEL, PENT_OPT_WINDOW_WARPS, PENT_OPT_WINDOWS, PENT_OPT_WINDOW_ROWS, PENT_OPT_PERSISTENT, PENT_OPT_FP64_INTERIOR, PENT_OPT_WINDOW_FORM,
                   PENT_OPT_PARTITION_ROWS, PENT_OPT_PERIODIC, PENT_OPT_REFINE_TOL_LOG2, PENT_OPT_RESIDUAL, PENT_OPT_ROWS_PER_THREAD,
                   PENT_OPT_THREADS_PER_SYSTEM,
                   PENT_OPT_UNROLL, PENT_RESIDUAL_F64,
                   PENT_RESIDUAL_FF, PentError, check)

__all__ = ["Plan", "PentError", "PENT_F64", "PENT_F32_REFINE", "PENT_RESIDUAL_FF", "PENT_RESIDUAL_F64",
           "library_path", "load_library", "window_layout", "system_window_layout", "adi_plans_factor", "adi_step_2d", "adi_steps_2d", "ADI2D"]

__version__ = "0.1.0"


def library_path():
    return _lib.LIB_PATH


def load_library():
    return _lib.load()


def _torch():
    import torch  # imported lazily: the CPU-only checks load the library without touching CUDA
    return torch


def _dev_ptr(t, what: str, dtype=None) -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (the library has no CPU path)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


class Plan:
    """A batch of pentadiagonal systems, factored once on the device.

    n:         int (every system has n rows) or a sequence of row counts.
    batch:     number of systems (required when n is an int).
    shared:    all systems share one matrix (band / sigma describe one system).
    precision: PENT_F64 or PENT_F32_REFINE.
    periodic:  cyclic systems (Sec. 2.3), solved by Navon's reduction (FP64, uniform n >= 5).
    """

    def __init__(self, n, batch: Optional[int] = None, shared: bool = False, precision: int = PENT_F64,
                 device=None, stream=None, tune_cache: Optional[str] = None, options: Optional[dict] = None,
                 periodic: bool = False):
        torch = _torch()
        L = _lib.load()
        self._L = L
        self._h = ctypes.c_void_p()
        if isinstance(n, int):
            if batch is None:
                raise ValueError("batch is required when n is an int")
            nptr, n_uniform = None, int(n)
            self.n = [int(n)] * int(batch)
        else:
            ns = [int(v) for v in n]
            if batch is not None and batch != len(ns):
                raise ValueError("batch does not match len(n)")
            batch = len(ns)
            self._narr = (ctypes.c_int64 * batch)(*ns)
            nptr, n_uniform = self._narr, 0
            self.n = ns
        self.batch = int(batch)
        self.shared = bool(shared)
        self.precision = int(precision)
        self.rows = sum(self.n)
        check(L.pent_plan_create(ctypes.byref(self._h), self.batch, nptr, n_uniform, int(self.shared),
                                 self.precision, tune_cache.encode() if tune_cache else None), "pent_plan_create")
        options = dict(options or {})
        if periodic:
            options[PENT_OPT_PERIODIC] = 1
        self.periodic = bool(periodic)
        for key, value in options.items():  # layout options must precede pent_plan_bind
            check(L.pent_plan_set_option(self._h, int(key), int(value)), "pent_plan_set_option")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = int(L.pent_plan_workspace_bytes(self._h))
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        check(L.pent_plan_bind(self._h, self.workspace.data_ptr(), ctypes.c_void_p(self.stream.cuda_stream)),
              "pent_plan_bind")

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.pent_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def workspace_bytes(self) -> int:
        return int(self._L.pent_plan_workspace_bytes(self._h))

    # -- options
    def set_option(self, key: int, value: int):
        check(self._L.pent_plan_set_option(self._h, key, int(value)), "pent_plan_set_option")

    def get_option(self, key: int) -> int:
        v = ctypes.c_int64()
        check(self._L.pent_plan_get_option(self._h, key, ctypes.byref(v)), "pent_plan_get_option")
        return int(v.value)

    def system_config(self, system: int) -> tuple:
        """(rows per thread, threads per system) for FP32+refine, (unroll, warps per CTA) for FP64."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        check(self._L.pent_plan_system_config(self._h, int(system), ctypes.byref(a), ctypes.byref(b)),
              "pent_plan_system_config")
        return int(a.value), int(b.value)

    # -- factorisation
    def factor(self, a, b, c, d, e):
        """Factor general bands (device float64 tensors, system-major)."""
        torch = _torch()
        ptrs = [_dev_ptr(t, name, torch.float64) for t, name in zip((a, b, c, d, e), "abcde")]
        check(self._L.pent_factor_batch(self._h, *ptrs), "pent_factor_batch")

    def factor_hyperdiff(self, sigma):
        """Factor A_s = I + sigma_s D4 (no-flux) from device float64 sigma."""
        torch = _torch()
        self._sigma_ref = sigma
        check(self._L.pent_factor_hyperdiff(self._h, _dev_ptr(sigma, "sigma", torch.float64)), "pent_factor_hyperdiff")

    def refactor_solve(self, sigma, f, x=None):
        """Factor A_s = I + sigma_s D4 from a new sigma and solve A_s x = f in one call (the matrix
        changes every step); the plan stays factored with the new sigma."""
        torch = _torch()
        if x is None:
            x = torch.empty_like(f)
        self._sigma_ref = sigma
        check(self._L.pent_refactor_solve_hyperdiff(self._h, _dev_ptr(sigma, "sigma", torch.float64),
                                                    _dev_ptr(f, "f", torch.float64), _dev_ptr(x, "x", torch.float64)),
              "pent_refactor_solve_hyperdiff")
        return x

    # -- solves
    def solve(self, f, x=None, max_refine: int = 2):
        """x_s = A_s^{-1} f_s; x may be f (in place)."""
        torch = _torch()
        if x is None:
            x = torch.empty_like(f)
        check(self._L.pent_solve_batch(self._h, _dev_ptr(f, "f", torch.float64), _dev_ptr(x, "x", torch.float64),
                                       int(max_refine)), "pent_solve_batch")
        return x

    def solve_host(self, f_host, x_host, f_dev=None, x_dev=None, max_refine: int = 2, chunks: int = 16,
                   direct: bool = False):
        """Solve for right-hand sides held in pinned host memory: the library copies f to the
        device staging buffer, solves and copies x back, in `chunks` slices whose copies and
        solves overlap (pent_solve_host_batch); asynchronous on the plan's stream.  f_dev / x_dev
        are device staging buffers (allocated here if not given; x_dev may be f_dev).
        direct=True (FP32+refine plans): no staging; the solve kernels read f_host and write
        x_host in place over the host link (x_host may be f_host); both must be pinned."""
        torch = _torch()
        if f_host.is_cuda or x_host.is_cuda:
            raise ValueError("solve_host takes host tensors")
        for t, name in ((f_host, "f_host"), (x_host, "x_host")):
            if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != self.rows:
                raise ValueError(f"{name} must be a contiguous float64 tensor of {self.rows} elements")
        if direct:
            if f_dev is not None or x_dev is not None:
                raise ValueError("direct solves take no staging buffers")
            if not (f_host.is_pinned() and x_host.is_pinned()):
                raise ValueError("direct solves need pinned host tensors")
            self._host_refs = (f_host, x_host)
            check(self._L.pent_solve_host_batch(self._h, f_host.data_ptr(), x_host.data_ptr(), None, None,
                                                int(chunks), int(max_refine)), "pent_solve_host_batch")
            return x_host
        fd = f_dev if f_dev is not None else torch.empty(self.rows, dtype=torch.float64, device=self.device)
        xd = x_dev if x_dev is not None else torch.empty_like(fd)
        self._host_refs = (f_host, x_host, fd, xd)
        check(self._L.pent_solve_host_batch(self._h, f_host.data_ptr(), x_host.data_ptr(),
                                            _dev_ptr(fd, "f_dev", torch.float64), _dev_ptr(xd, "x_dev", torch.float64),
                                            int(chunks), int(max_refine)), "pent_solve_host_batch")
        return x_host

    def solve_steps(self, x, nsteps: int, max_refine: int = 2):
        """nsteps in-place implicit steps x <- A^{-1} x (one CUDA graph)."""
        torch = _torch()
        check(self._L.pent_solve_steps(self._h, _dev_ptr(x, "x", torch.float64), int(nsteps), int(max_refine)),
              "pent_solve_steps")
        return x

    def step(self, C, mu=None, nu=None, nsteps: int = 1, max_refine: int = 2):
        """nsteps semi-implicit steps in place: A_s C <- C + mu_s D2(C^3 - C) - nu_s D4 C, the right-hand
        side assembled inside the solve kernel (Cahn-Hilliard: mu = D dt/dx^2; Crank-Nicolson
        hyperdiffusion: nu = sigma).  mu, nu: device float64 tensors of one value per system (one when
        the matrix is shared) or None for zero.  Several steps run as one CUDA graph.  max_refine: the
        refinement steps of a PENT_F32_REFINE plan (the right-hand side is then assembled in
        float-float arithmetic)."""
        torch = _torch()
        mp = _dev_ptr(mu, "mu", torch.float64) if mu is not None else None
        np_ = _dev_ptr(nu, "nu", torch.float64) if nu is not None else None
        self._step_refs = (mu, nu)  # graphs keep the pointers
        check(self._L.pent_step_batch(self._h, mp, np_, _dev_ptr(C, "C", torch.float64), int(nsteps),
                                      int(max_refine)), "pent_step_batch")
        return C

    def adjoint_solve(self, f, x=None, max_refine: int = 2):
        """y_s = A_s^{-T} f_s from the stored factors (for matrices built from sigma, which are
        symmetric, by the solve itself; max_refine as in solve)."""
        torch = _torch()
        if x is None:
            x = torch.empty_like(f)
        check(self._L.pent_adjoint_solve_batch(self._h, _dev_ptr(f, "f", torch.float64),
                                               _dev_ptr(x, "x", torch.float64), int(max_refine)),
              "pent_adjoint_solve_batch")
        return x

    def sigma_grad(self, mu, x, g_sigma):
        """g_sigma[s] -= mu_s . (D4 x_s)."""
        torch = _torch()
        check(self._L.pent_hyperdiff_sigma_grad(self._h, _dev_ptr(mu, "mu", torch.float64),
                                                _dev_ptr(x, "x", torch.float64),
                                                _dev_ptr(g_sigma, "g_sigma", torch.float64)),
              "pent_hyperdiff_sigma_grad")
        return g_sigma

    # -- diagnostics
    def info(self):
        """(status, bad_system, bad_row, refine_steps_used); synchronises the stream."""
        bs, br, rs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        st = self._L.pent_get_info(self._h, ctypes.byref(bs), ctypes.byref(br), ctypes.byref(rs))
        return int(st), int(bs.value), int(br.value), int(rs.value)

    def clear_info(self):
        check(self._L.pent_clear_info(self._h), "pent_clear_info")


def adi_step_2d(px: Plan, py: Plan, C, gamma: float, dt: float, dx: float, max_refine: int = 0):
    torch = _torch()
    ny, nx = C.shape
    check(_lib.load().adi_step_2d(px._h, py._h, _dev_ptr(C, "C", torch.float64), nx, ny, float(gamma), float(dt),
                                  float(dx), int(max_refine)), "adi_step_2d")
    return C


def window_layout(n: int, window_rows: int, overlap: int):
    """The windows of an n-row system (pent_window_layout): an int32 array of rows (first row,
    rows, first kept, end kept), the kept rows relative to the window; empty when n fits one CTA."""
    import numpy as np
    L = _lib.load()
    cnt = int(L.pent_window_layout(int(n), int(window_rows), int(overlap), None, 0))
    out = np.zeros((max(cnt, 0), 4), dtype=np.int32)
    if cnt > 0:
        L.pent_window_layout(int(n), int(window_rows), int(overlap), out.ctypes.data_as(ctypes.c_void_p), cnt)
    return out


def system_window_layout(n: int, window_rows: int, overlap: int):
    """The FP64 system windows of an n-row system (pent_system_window_layout): an int32 array of
    rows (first row walked, first kept, end kept), one window for n <= window_rows."""
    import numpy as np
    L = _lib.load()
    cnt = int(L.pent_system_window_layout(int(n), int(window_rows), int(overlap), None, 0))
    out = np.zeros((max(cnt, 0), 3), dtype=np.int32)
    if cnt > 0:
        L.pent_system_window_layout(int(n), int(window_rows), int(overlap), out.ctypes.data_as(ctypes.c_void_p), cnt)
    return out


def adi_plans_factor(px: Plan, py: Plan, gamma: float, dt: float, dx: float):
    """Factor both plans of an ADI step for (gamma, dt, dx) (see adi_step_2d)."""
    check(_lib.load().adi_plans_factor(px._h, py._h, float(gamma), float(dt), float(dx)), "adi_plans_factor")


def adi_steps_2d(px: Plan, py: Plan, C, gamma: float, dt: float, dx: float, nsteps: int, max_refine: int = 0):
    torch = _torch()
    ny, nx = C.shape
    check(_lib.load().adi_steps_2d(px._h, py._h, _dev_ptr(C, "C", torch.float64), nx, ny, float(gamma), float(dt),
                                   float(dx), int(max_refine), int(nsteps)), "adi_steps_2d")
    return C


class ADI2D:
    """Alternating-direction Cahn-Hilliard stepper on an ny x nx no-flux grid.

    Two shared-matrix plans (n = nx for the row sweeps, n = ny for the column
    sweeps), factored once by adi_plans_factor for (gamma, dt, dx), which also
    derives the scheme's coefficients; `step` advances a device field C
    (ny x nx, float64, in place).
    """

    def __init__(self, nx: int, ny: int, gamma: float, dt: float, dx: float, device=None, stream=None):
        self.nx, self.ny = int(nx), int(ny)
        self.gamma, self.dt, self.dx = float(gamma), float(dt), float(dx)
        self.px = Plan(self.nx, batch=self.ny, shared=True, device=device, stream=stream)
        self.py = Plan(self.ny, batch=self.nx, shared=True, device=self.px.device, stream=self.px.stream)
        check(_lib.load().adi_plans_factor(self.px._h, self.py._h, self.gamma, self.dt, self.dx), "adi_plans_factor")

    def step(self, C, nsteps: int = 1):
        if tuple(C.shape) != (self.ny, self.nx):
            raise ValueError(f"C must have shape ({self.ny}, {self.nx})")
        if nsteps == 1:
            return adi_step_2d(self.px, self.py, C, self.gamma, self.dt, self.dx)
        return adi_steps_2d(self.px, self.py, C, self.gamma, self.dt, self.dx, nsteps)

    def info(self):
        return self.px.info(), self.py.info()
