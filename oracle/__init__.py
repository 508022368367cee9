"""CPU oracle for the batched pentadiagonal solver (test infrastructure only).

The oracle is plain serial FP64 C (`pent_oracle.c`) reached through ctypes.
It restates the method of Gloster, O Naraigh and Pang (arXiv 1807.07382):
the pentadiagonal LU factorisation without pivoting and the forward and back
substitutions of Sec. 2.4, the hyperdiffusion band of Sec. 2.2-2.3 (with the
no-flux reading documented in the C file), the adjoint solve as the plain
solve of the transposed system, and the 2D alternating-direction step named
in Sec. 4.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The CUDA library and its Python binding
never import it; the two share no code.

Periodic systems (Sec. 2.3) are solved by Navon's reduction as the paper
states it: the last two unknowns from the 2x2 system of Eq. (first_two), then
the rest from Eq. (solve).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pent_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libpent_oracle.so"
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"libpent_oracle.{os.getpid()}.so"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", str(tmp), str(_SRC), "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(str(path))
            L.po_max_threads.restype = ctypes.c_int
            L.po_band_d4.argtypes = [_i64] + [_dp] * 5
            L.po_band_hyperdiff.argtypes = [_i64, ctypes.c_double] + [_dp] * 5
            L.po_factor.argtypes = [_i64] + [_dp] * 10
            L.po_factor.restype = _i64
            L.po_solve.argtypes = [_i64] + [_dp] * 8
            L.po_transpose_band.argtypes = [_i64] + [_dp] * 10
            L.po_matvec.argtypes = [_i64] + [_dp] * 7
            L.po_factor_batch.argtypes = [_i64, _ip] + [_dp] * 10 + [ctypes.c_int, _ip]
            L.po_factor_batch.restype = _i64
            L.po_solve_batch.argtypes = [_i64, _ip] + [_dp] * 7 + [ctypes.c_int]
            L.po_adjoint_solve.argtypes = [_i64] + [_dp] * 8
            L.po_adjoint_solve.restype = _i64
            L.po_adjoint_solve_batch.argtypes = [_i64, _ip] + [_dp] * 7 + [ctypes.c_int]
            L.po_adjoint_solve_batch.restype = _i64
            L.po_hyperdiff_steps.argtypes = [_i64, _ip, _dp, ctypes.c_int, _i64, _dp, ctypes.c_int]
            L.po_hyperdiff_steps.restype = _i64
            L.po_laplacian_noflux.argtypes = [_i64, _i64, _dp, _dp]
            L.po_ch_rhs.argtypes = [_i64, _i64, _dp, ctypes.c_double, ctypes.c_double, _dp]
            L.po_adi_step.argtypes = [_i64, _i64, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int]
            L.po_adi_step.restype = _i64
            L.po_adi_solve.argtypes = [_i64, _i64, _dp, ctypes.c_double, ctypes.c_int]
            L.po_adi_solve.restype = _i64
            L.po_adi_step_ms.argtypes = [_i64, _i64, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.po_adi_step_ms.restype = _i64
            L.po_hyperdiff_loss_grad.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _dp, _dp, ctypes.c_int]
            L.po_hyperdiff_loss_grad.restype = ctypes.c_double
            L.po_hyperdiff_vjp.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _dp, _dp, ctypes.c_int]
            L.po_periodic_matvec.argtypes = [_i64] + [_dp] * 7
            L.po_band_periodic_hyperdiff.argtypes = [_i64, ctypes.c_double] + [_dp] * 5
            L.po_periodic_cn_rhs.argtypes = [_i64, ctypes.c_double, _dp, _dp]
            L.po_periodic_solve.argtypes = [_i64] + [_dp] * 7
            L.po_periodic_solve.restype = _i64
            L.po_periodic_solve_batch.argtypes = [_i64, _i64] + [_dp] * 7 + [ctypes.c_int]
            L.po_periodic_solve_batch.restype = _i64
            L.po_periodic_steps.argtypes = [_i64, _i64, _dp, ctypes.c_int, _i64, ctypes.c_int, _dp, ctypes.c_int]
            L.po_periodic_steps.restype = _i64
            L.po_explicit_rhs.argtypes = [_i64, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            L.po_explicit_steps.argtypes = [_i64, _ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, _i64, _dp,
                                            ctypes.c_int]
            L.po_explicit_steps.restype = _i64
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _pi(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_ip)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().po_max_threads())


def offsets(n) -> np.ndarray:
    n = np.asarray(n, dtype=np.int64).reshape(-1)
    off = np.zeros(n.shape[0] + 1, dtype=np.int64)
    np.cumsum(n, out=off[1:])
    return off


# ----------------------------------------------------------------------------- bands

def band_d4(n: int):
    """Band (a, b, c, d, e) of the no-flux fourth difference D4 = D2N^2."""
    out = [np.zeros(n) for _ in range(5)]
    lib().po_band_d4(n, *[_p(o) for o in out])
    return tuple(out)


def band_hyperdiff(n: int, sigma: float):
    """Band of A = I + sigma * D4 (no-flux, cell-centred)."""
    out = [np.zeros(n) for _ in range(5)]
    lib().po_band_hyperdiff(n, float(sigma), *[_p(o) for o in out])
    return tuple(out)


def band_hyperdiff_batch(n_per_system, sigma):
    """Concatenated bands of A_s = I + sigma_s D4 for systems of sizes n_per_system."""
    n_per_system = np.asarray(n_per_system, dtype=np.int64).reshape(-1)
    sigma = np.broadcast_to(np.asarray(sigma, dtype=np.float64), n_per_system.shape)
    parts = [band_hyperdiff(int(n), float(s)) for n, s in zip(n_per_system, sigma)]
    return tuple(np.concatenate([p[k] for p in parts]) if parts else np.zeros(0) for k in range(5))


def matvec(band, x):
    n = x.shape[0]
    y = np.zeros(n)
    lib().po_matvec(n, *[_p(_f64(b)) for b in band], _p(_f64(x)), _p(y))
    return y


def transpose_band(band):
    n = band[0].shape[0]
    out = [np.zeros(n) for _ in range(5)]
    lib().po_transpose_band(n, *[_p(_f64(b)) for b in band], *[_p(o) for o in out])
    return tuple(out)


# ----------------------------------------------------------------------------- factor / solve

def factor(band):
    """Factors (alpha, beta, gamma, delta, eps) of one system, and the first failing row or -1."""
    n = band[0].shape[0]
    out = [np.zeros(n) for _ in range(5)]
    r = lib().po_factor(n, *[_p(_f64(b)) for b in band], *[_p(o) for o in out])
    return tuple(out), int(r)


def solve(factors, f):
    n = f.shape[0]
    x = np.zeros(n)
    g = np.zeros(n)
    lib().po_solve(n, *[_p(_f64(v)) for v in factors], _p(_f64(f)), _p(x), _p(g))
    return x


def factor_batch(n_per_system, band, nthreads: int = 0):
    off = offsets(n_per_system)
    m = int(off[-1])
    out = [np.zeros(m) for _ in range(5)]
    bad_row = np.zeros(1, dtype=np.int64)
    bad = lib().po_factor_batch(len(off) - 1, _pi(off), *[_p(_f64(b)) for b in band], *[_p(o) for o in out],
                                nthreads, _pi(bad_row))
    return tuple(out), int(bad), int(bad_row[0])


def solve_batch(n_per_system, factors, f, nthreads: int = 0):
    off = offsets(n_per_system)
    x = np.zeros(int(off[-1]))
    lib().po_solve_batch(len(off) - 1, _pi(off), *[_p(_f64(v)) for v in factors], _p(_f64(f)), _p(x), nthreads)
    return x


def adjoint_solve_batch(n_per_system, band, f, nthreads: int = 0):
    """y_s = A_s^{-T} f_s from the band of A (transposed band, factored and solved)."""
    off = offsets(n_per_system)
    y = np.zeros(int(off[-1]))
    bad = lib().po_adjoint_solve_batch(len(off) - 1, _pi(off), *[_p(_f64(b)) for b in band], _p(_f64(f)), _p(y),
                                       nthreads)
    if bad >= 0:
        raise ArithmeticError(f"transposed factorisation failed in system {bad}")
    return y


def hyperdiff_steps(n_per_system, sigma, field0, steps: int, shared: bool = False, nthreads: int = 0):
    """`steps` implicit hyperdiffusion steps on every system; returns the new field."""
    off = offsets(n_per_system)
    field = np.array(field0, dtype=np.float64, copy=True)
    sig = _f64(np.asarray(sigma, dtype=np.float64).reshape(-1))
    bad = lib().po_hyperdiff_steps(len(off) - 1, _pi(off), _p(sig), int(bool(shared)), int(steps), _p(field),
                                   nthreads)
    if bad >= 0:
        raise ArithmeticError(f"factorisation failed in system {bad}")
    return field


# ----------------------------------------------------------------------------- 2D

def laplacian_noflux(v):
    v = _f64(v)
    out = np.zeros_like(v)
    ny, nx = v.shape
    lib().po_laplacian_noflux(nx, ny, _p(v), _p(out))
    return out


def ch_rhs(C, mu: float, sigma: float):
    C = _f64(C)
    out = np.zeros_like(C)
    ny, nx = C.shape
    lib().po_ch_rhs(nx, ny, _p(C), float(mu), float(sigma), _p(out))
    return out


def adi_solve(rhs, sigma: float, nthreads: int = 0):
    """dC with (I + sigma D4_x)(I + sigma D4_y) dC = rhs (x sweep, then y sweep)."""
    r = np.array(rhs, dtype=np.float64, copy=True)
    ny, nx = r.shape
    st = lib().po_adi_solve(nx, ny, _p(r), float(sigma), nthreads)
    if st >= 0:
        raise ArithmeticError(f"ADI factorisation failed in direction {st}")
    return r


def adi_step_ms(C, mu: float, sigma: float, nthreads: int = 0):
    C = np.array(C, dtype=np.float64, copy=True)
    ny, nx = C.shape
    st = lib().po_adi_step_ms(nx, ny, _p(C), float(mu), float(sigma), nthreads)
    if st >= 0:
        raise ArithmeticError(f"ADI factorisation failed in direction {st}")
    return C


def adi_step(C, gamma: float, dt: float, dx: float, nthreads: int = 0):
    C = np.array(C, dtype=np.float64, copy=True)
    ny, nx = C.shape
    st = lib().po_adi_step(nx, ny, _p(C), float(gamma), float(dt), float(dx), nthreads)
    if st >= 0:
        raise ArithmeticError(f"ADI factorisation failed in direction {st}")
    return C


# ----------------------------------------------------------------------------- loss / gradient

def hyperdiff_loss_grad(sigma, T: int, c0, target, nthreads: int = 0):
    """Loss sum_s ||x_s^T - target_s||^2 and its gradients w.r.t. C0 and sigma."""
    sigma = _f64(sigma)
    c0 = _f64(c0)
    target = _f64(target)
    batch, n = c0.shape
    gc = np.zeros_like(c0)
    gs = np.zeros(batch)
    loss = lib().po_hyperdiff_loss_grad(batch, n, _p(sigma), int(T), _p(c0), _p(target), _p(gc), _p(gs), nthreads)
    return float(loss), gc, gs


def hyperdiff_vjp(sigma, T: int, c0, lambda_T, nthreads: int = 0):
    """(dC0, dsigma) of the T-step map for a given lambda^T = dL/dx^T."""
    sigma = _f64(sigma)
    c0 = _f64(c0)
    lam = _f64(lambda_T)
    batch, n = c0.shape
    gc = np.zeros_like(c0)
    gs = np.zeros(batch)
    lib().po_hyperdiff_vjp(batch, n, _p(sigma), int(T), _p(c0), _p(lam), _p(gc), _p(gs), nthreads)
    return gc, gs


# ----------------------------------------------------------------------------- periodic (Sec. 2.3)

def band_periodic_hyperdiff(n: int, sigma: float):
    """Cyclic band of Eq. (matrix_sys): a = e = sigma, b = d = -4 sigma, c = 1 + 6 sigma."""
    out = [np.zeros(n) for _ in range(5)]
    lib().po_band_periodic_hyperdiff(n, float(sigma), *[_p(o) for o in out])
    return tuple(out)


def periodic_matvec(band, x):
    """y = A x for a cyclic band (column indices modulo n)."""
    x = _f64(x)
    y = np.zeros_like(x)
    lib().po_periodic_matvec(x.shape[0], *[_p(_f64(b)) for b in band], _p(x), _p(y))
    return y


def periodic_cn_rhs(sigma: float, C):
    """Crank-Nicolson right-hand side of Eq. (matrix_sys), periodic."""
    C = _f64(C)
    f = np.zeros_like(C)
    lib().po_periodic_cn_rhs(C.shape[0], float(sigma), _p(C), _p(f))
    return f


def periodic_solve(band, f):
    """x = A^{-1} f for one cyclic system by Navon's reduction; raises on a failed pivot."""
    f = _f64(f)
    x = np.zeros_like(f)
    r = lib().po_periodic_solve(f.shape[0], *[_p(_f64(b)) for b in band], _p(f), _p(x))
    if r >= 0:
        raise ArithmeticError(f"periodic reduction failed at row {r}")
    return x


def periodic_solve_row(band, f) -> int:
    """The failing row of the reduction (-1 if none)."""
    f = _f64(f)
    x = np.zeros_like(f)
    return int(lib().po_periodic_solve(f.shape[0], *[_p(_f64(b)) for b in band], _p(f), _p(x)))


def periodic_solve_batch(n: int, band, f, nthreads: int = 0):
    """Cyclic solve for every system of a batch of n-row systems (system-major)."""
    f = _f64(f)
    x = np.zeros_like(f)
    bad = lib().po_periodic_solve_batch(f.shape[0] // n, n, *[_p(_f64(b)) for b in band], _p(f), _p(x), nthreads)
    if bad >= 0:
        raise ArithmeticError(f"periodic reduction failed in system {bad}")
    return x


def periodic_steps(n: int, sigma, field0, steps: int, cn: bool = True, shared: bool = False, nthreads: int = 0):
    """`steps` periodic hyperdiffusion steps (Crank-Nicolson or implicit Euler) on every system."""
    field = np.array(field0, dtype=np.float64, copy=True)
    sig = _f64(np.asarray(sigma, dtype=np.float64).reshape(-1))
    bad = lib().po_periodic_steps(field.shape[0] // n, n, _p(sig), int(bool(shared)), int(steps), int(bool(cn)),
                                  _p(field), nthreads)
    if bad >= 0:
        raise ArithmeticError(f"periodic reduction failed in system {bad}")
    return field


# ----------------------------------------------------------------------------- steps with an explicit part

def explicit_rhs(C, mu: float, nu: float, periodic: bool = False):
    """f = C + mu D2(C^3 - C) - nu D4 C on the no-flux (reflected) or periodic grid."""
    C = _f64(C)
    f = np.zeros_like(C)
    u = np.zeros_like(C)
    lib().po_explicit_rhs(C.shape[0], int(bool(periodic)), float(mu), float(nu), _p(C), _p(f), _p(u))
    return f


def explicit_steps(n_per_system, sigma, mu, nu, field0, steps: int, periodic: bool = False, shared: bool = False,
                   nthreads: int = 0):
    """`steps` steps (I + sigma_s D4) C^{k+1} = C^k + mu_s D2(C^3 - C)^k - nu_s D4 C^k on every system.
    mu or nu may be None (zero)."""
    off = offsets(n_per_system)
    field = np.array(field0, dtype=np.float64, copy=True)
    sig = _f64(np.asarray(sigma, dtype=np.float64).reshape(-1))
    m_ = None if mu is None else _f64(np.asarray(mu, dtype=np.float64).reshape(-1))
    n_ = None if nu is None else _f64(np.asarray(nu, dtype=np.float64).reshape(-1))
    bad = lib().po_explicit_steps(len(off) - 1, _pi(off), int(bool(periodic)), _p(sig),
                                  _p(m_) if m_ is not None else None, _p(n_) if n_ is not None else None,
                                  int(bool(shared)), int(steps), _p(field), nthreads)
    if bad >= 0:
        raise ArithmeticError(f"factorisation failed in system {bad}")
    return field
