"""Seeded synthetic inputs for the batched pentadiagonal workloads.

This module is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark. It holds only random-number generation and the *shapes* of the inputs
(sizes, value ranges, initial fields); it contains none of the solver's
arithmetic (no band, no factorisation, no substitution, no time step).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Its k-th output from seed s is
mix(s + (k+1)*0x9E3779B97F4A7C15), so the generator is counter-based and any
range of draws can be produced directly.  A double in [0, 1) is (u >> 11) * 2^-53.

Workloads (the paper's hyperdiffusion batches, Sec. 3, and the 2D ADI extension
named in Sec. 4), each drawn from seed BASE_SEED + index:

  0  64 systems, N=256, shared sigma=0.5, 4 cosine modes + U[-0.01,0.01], 100 steps
  1  65,536 systems, N=1024, sigma_i log-U[1e-3,10], C0 U[-1,1], 1,000 steps
  2  2048 x 2048 Cahn-Hilliard ADI field, C0 U[-0.1,0.1], 500 steps
  3  20,000 systems, N log-U[64,16384], sigma_i log-U[1e-2,10], RHS U[-1,1], 200 steps
  4  4,096 systems, N=1024, sigma_i log-U[1e-3,10], C0 U[-1,1], T=50
  5  periodic Crank-Nicolson batch: 65,536 systems, N=512, one shared sigma_x = dt/(2 dx^4)
     with dt = 1e-8, dx = 1/N (the paper's validation parameters), C0 U[-1,1], 250 steps
  6  1D Cahn-Hilliard parameter batch: 65,536 systems, N=1024, sigma_i log-U[1e-3,10],
     mu_i log-U[1e-4,1e-1], C0 U[-1,1], 200 steps

Draw order inside one seed: per-system scalars first (sigma, then N where
present), then the field, system-major.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

BASE_SEED = 1807073820
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with `seed` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, count, _CHUNK):
            hi = min(count, lo + _CHUNK)
            k = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            z = s + k * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            out[lo:hi] = z ^ (z >> np.uint64(31))
    return out


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): (u >> 11) * 2^-53."""
    u = splitmix64(seed, start, count)
    return (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, start: int, count: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, start, count)


def log_uniform(seed: int, start: int, count: int, lo: float, hi: float) -> np.ndarray:
    u = uniform01(seed, start, count)
    return np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


@dataclass
class Workload1D:
    """A batch of 1D systems A_s x = f_s with A_s = I + sigma_s * D4 (no-flux)."""
    name: str
    n: np.ndarray            # int64 [batch], rows per system
    sigma: np.ndarray        # float64 [batch] (or [1] if shared)
    field0: np.ndarray       # float64 [sum(n)], system-major, initial field / RHS
    steps: int
    shared: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return int(self.n.shape[0])

    @property
    def offsets(self) -> np.ndarray:
        off = np.zeros(self.batch + 1, dtype=np.int64)
        np.cumsum(self.n, out=off[1:])
        return off

    @property
    def rows(self) -> int:
        return int(self.n.sum())


@dataclass
class Workload2D:
    name: str
    nx: int
    ny: int
    gamma: float
    dt: float
    dx: float
    field0: np.ndarray       # float64 [ny, nx], row-major
    steps: int


def hyperdiff_cosines(batch: int = 64, n: int = 256, steps: int = 100, seed_index: int = 0) -> Workload1D:
    """Shared sigma=0.5; C0 = sum of modes k in {1,2,3,5} with amplitudes
    {1, 0.5, 0.25, 0.125} on the cell-centred grid cos(pi k (i+1/2)/N),
    plus U[-0.01, 0.01] noise."""
    seed = BASE_SEED + seed_index
    i = np.arange(n, dtype=np.float64)
    base = np.zeros(n)
    for k, amp in zip((1, 2, 3, 5), (1.0, 0.5, 0.25, 0.125)):
        base += amp * np.cos(np.pi * k * (i + 0.5) / n)
    noise = uniform(seed, 0, batch * n, -0.01, 0.01).reshape(batch, n)
    f0 = (base[None, :] + noise).reshape(-1)
    return Workload1D("hyperdiff_cosines", np.full(batch, n, np.int64), np.array([0.5]), f0, steps, shared=True)


def hyperdiff_parametric(batch: int = 65536, n: int = 1024, steps: int = 1000, seed_index: int = 1,
                         sigma_range=(1e-3, 10.0)) -> Workload1D:
    """Per-system sigma_i log-uniform in [1e-3, 10]; C0 uniform in [-1, 1]."""
    seed = BASE_SEED + seed_index
    sigma = log_uniform(seed, 0, batch, *sigma_range)
    f0 = uniform(seed, batch, batch * n, -1.0, 1.0)
    return Workload1D("hyperdiff_parametric", np.full(batch, n, np.int64), sigma, f0, steps)


def ch_adi(nx: int = 2048, ny: int = 2048, steps: int = 500, seed_index: int = 2, gamma: float = 0.01,
           dt: float = 1e-6, length: float = 1.0) -> Workload2D:
    """C0 uniform in [-0.1, 0.1] on an ny x nx grid with dx = length / nx."""
    seed = BASE_SEED + seed_index
    f0 = uniform(seed, 0, nx * ny, -0.1, 0.1).reshape(ny, nx)
    return Workload2D("ch_adi", nx, ny, gamma, dt, length / nx, f0, steps)


def uneven(batch: int = 20000, steps: int = 200, seed_index: int = 3, n_range=(64, 16384),
           sigma_range=(1e-2, 10.0)) -> Workload1D:
    """N_s log-uniform in [64, 16384] (floored), sigma_s log-uniform in [1e-2, 10], RHS uniform in [-1, 1]."""
    seed = BASE_SEED + seed_index
    sigma = log_uniform(seed, 0, batch, *sigma_range)
    nf = log_uniform(seed, batch, batch, float(n_range[0]), float(n_range[1]))
    n = np.minimum(np.floor(nf).astype(np.int64), n_range[1])
    rows = int(n.sum())
    f0 = uniform(seed, 2 * batch, rows, -1.0, 1.0)
    return Workload1D("uneven", n, sigma, f0, steps)


def adjoint_batch(batch: int = 4096, n: int = 1024, steps: int = 50, seed_index: int = 4,
                  perturb: float = 0.01) -> Workload1D:
    """sigma_i log-uniform in [1e-3, 10], C0 uniform in [-1, 1]; the loss target is the
    forward solution at sigma_i * (1 + perturb)."""
    w = hyperdiff_parametric(batch, n, steps, seed_index)
    w.name = "adjoint"
    w.extra["perturb"] = perturb
    return w


def periodic_cn(batch: int = 65536, n: int = 512, steps: int = 250, seed_index: int = 5,
                dt: float = 1e-8, length: float = 1.0) -> Workload1D:
    """Shared sigma_x = dt / (2 dx^4), dx = length / n; C0 uniform in [-1, 1]."""
    seed = BASE_SEED + seed_index
    dx = length / n
    f0 = uniform(seed, 0, batch * n, -1.0, 1.0)
    return Workload1D("periodic_cn", np.full(batch, n, np.int64), np.array([dt / (2 * dx ** 4)]), f0, steps,
                      shared=True)


def ch_batch(batch: int = 65536, n: int = 1024, steps: int = 200, seed_index: int = 6,
             sigma_range=(1e-3, 10.0), mu_range=(1e-4, 1e-1)) -> Workload1D:
    """Per-system sigma_i log-uniform in [1e-3, 10] and mu_i log-uniform in [1e-4, 1e-1]
    (extra["mu"]); C0 uniform in [-1, 1]."""
    seed = BASE_SEED + seed_index
    sigma = log_uniform(seed, 0, batch, *sigma_range)
    mu = log_uniform(seed, batch, batch, *mu_range)
    f0 = uniform(seed, 2 * batch, batch * n, -1.0, 1.0)
    return Workload1D("ch_batch", np.full(batch, n, np.int64), sigma, f0, steps, extra={"mu": mu})


def random_bands(batch: int, n: int, seed: int, kind: str = "diagdom") -> tuple:
    """Random pentadiagonal bands (a, b, c, d, e), each float64 [batch*n].

    kind="diagdom": off-diagonals U[-1,1], c = 1 + sum|off| + U[0,1] (strictly
    row diagonally dominant, not symmetric).
    kind="spd": symmetric, built as B B^T + n I style shift is avoided; instead
    c = 4.5 + U[0,1] with symmetric off-diagonals in U[-1,1] (diagonally dominant,
    hence SPD).
    """
    m = batch * n
    if kind == "diagdom":
        a, b, d, e = (uniform(seed, k * m, m, -1.0, 1.0) for k in range(4))
        c = 1.0 + np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e) + uniform01(seed, 4 * m, m)
        return a, b, c, d, e
    if kind == "spd":
        d = uniform(seed, 0, m, -1.0, 1.0).reshape(batch, n)
        e = uniform(seed, m, m, -1.0, 1.0).reshape(batch, n)
        b = np.zeros_like(d)
        a = np.zeros_like(e)
        b[:, 1:] = d[:, :-1]
        a[:, 2:] = e[:, :-2]
        c = 4.5 + uniform01(seed, 2 * m, m).reshape(batch, n)
        return a.reshape(-1), b.reshape(-1), c.reshape(-1), d.reshape(-1), e.reshape(-1)
    raise ValueError(kind)
