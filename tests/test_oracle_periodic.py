"""Pins for the oracle's periodic systems (Sec. 2.3, Navon's reduction): a dense
library solve of the full cyclic matrix, the circulant's exact eigenmodes under
the Crank-Nicolson and implicit steps, mass conservation, and the convergence
exponent the paper prints for this very scheme (Sec. 2.5, Fig. 2).  No GPU."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_cyclic(band):
    """Dense n x n matrix: row i = a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1} + e_i x_{i+2}, mod n."""
    a, b, c, d, e = band
    n = len(c)
    A = np.zeros((n, n))
    for i in range(n):
        for off, v in ((-2, a), (-1, b), (0, c), (1, d), (2, e)):
            A[i, (i + off) % n] += v[i]
    return A


def d4_circulant(n):
    D = np.zeros((n, n))
    for i in range(n):
        for off, w in ((-2, 1), (-1, -4), (0, 6), (1, -4), (2, 1)):
            D[i, (i + off) % n] += w
    return D


def symmetric_cyclic_band(n, seed):
    """Random symmetric cyclic band, diagonally dominant (hence SPD): d_i = b_{i+1}, e_i = a_{i+2} mod n."""
    d = synth.uniform(seed, 0, n, -1, 1)
    e = synth.uniform(seed, n, n, -1, 1)
    b = np.roll(d, 1)   # b_i = d_{i-1}
    a = np.roll(e, 2)   # a_i = e_{i-2}
    c = 4.5 + synth.uniform01(seed, 2 * n, n)
    return a, b, c, d, e


def rel(x, ref):
    return np.max(np.abs(x - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("n", [5, 6, 7, 8, 9, 12, 33, 100, 257])
@pytest.mark.parametrize("kind", ["diagdom", "spd"])
def test_periodic_solve_matches_dense(n, kind):
    band = synth.random_bands(1, n, seed=300 + n, kind="diagdom") if kind == "diagdom" else \
        symmetric_cyclic_band(n, 400 + n)
    f = synth.uniform(500 + n, 0, n, -1, 1)
    x = oracle.periodic_solve(band, f)
    ref = np.linalg.solve(dense_cyclic(band), f)
    assert rel(x, ref) <= 1e-13


def test_periodic_matvec_is_the_cyclic_band():
    n = 11
    band = synth.random_bands(1, n, seed=9, kind="diagdom")
    x = synth.uniform(10, 0, n, -1, 1)
    assert np.allclose(oracle.periodic_matvec(band, x), dense_cyclic(band) @ x, rtol=0, atol=1e-14)


def test_periodic_band_is_the_paper_matrix():
    """Eq. (matrix_sys): a = e = sigma, b = d = -4 sigma, c = 1 + 6 sigma, with the corners of Eq. (matrix_sys1)."""
    n, s = 9, 0.37
    A = dense_cyclic(oracle.band_periodic_hyperdiff(n, s))
    assert np.array_equal(A, np.eye(n) + s * d4_circulant(n))
    assert A[0, n - 2] == s and A[0, n - 1] == -4 * s and A[n - 1, 0] == -4 * s and A[n - 1, 1] == s


def test_periodic_cn_rhs_is_the_paper_rhs():
    n, s = 10, 2.5
    C = synth.uniform(12, 0, n, -1, 1)
    assert np.allclose(oracle.periodic_cn_rhs(s, C), (np.eye(n) - s * d4_circulant(n)) @ C, rtol=0, atol=1e-13)


def test_periodic_batch_equals_single_solves():
    n, batch = 17, 6
    band = synth.random_bands(batch, n, seed=33, kind="diagdom")
    f = synth.uniform(34, 0, batch * n, -1, 1)
    x = oracle.periodic_solve_batch(n, band, f)
    for s in range(batch):
        sl = slice(s * n, (s + 1) * n)
        assert np.array_equal(x[sl], oracle.periodic_solve(tuple(v[sl] for v in band), f[sl]))


@pytest.mark.parametrize("cn", [True, False])
@pytest.mark.parametrize("k", [1, 3, 7])
def test_periodic_steps_mode_amplification(cn, k):
    """cos(2 pi k i / n) is an eigenvector of the circulant D4 with eigenvalue 16 sin^4(pi k / n):
    per step it is multiplied by (1 - s l)/(1 + s l) (Crank-Nicolson) or 1/(1 + s l)."""
    n, s, T = 64, 0.8, 40
    i = np.arange(n)
    lam = 16 * math.sin(math.pi * k / n) ** 4
    G = (1 - s * lam) / (1 + s * lam) if cn else 1 / (1 + s * lam)
    for mode in (np.cos(2 * math.pi * k * i / n), np.sin(2 * math.pi * k * i / n)):
        out = oracle.periodic_steps(n, [s], mode, T, cn=cn)
        assert np.max(np.abs(out - G ** T * mode)) <= 1e-13


def test_periodic_steps_conserve_mass():
    n, batch = 48, 5
    sig = synth.log_uniform(7, 0, batch, 1e-2, 1e3)
    C = synth.uniform(7, batch, batch * n, -1, 1)
    out = oracle.periodic_steps(n, sig, C, 25)
    for s in range(batch):
        sl = slice(s * n, (s + 1) * n)
        assert abs(out[sl].sum() - C[sl].sum()) <= 1e-12 * np.abs(C[sl]).sum()


def test_periodic_singular_schur_complement_is_reported():
    """A = circulant with rows [0, 0, 1, 0, 0] except a zero 2x2 trailing block: E = I, S = 0."""
    n = 6
    a, b, c, d, e = (np.zeros(n) for _ in range(5))
    c[:] = 1.0
    c[n - 2:] = 0.0
    assert oracle.periodic_solve_row((a, b, c, d, e), np.ones(n)) == n - 2


def test_periodic_convergence_exponent_matches_paper_fig2():
    """The paper's own validation (Sec. 2.5): periodic Crank-Nicolson with sigma_x = dt / (2 dx^4),
    C0 = cos(k x), k = 2 pi n / L, x_i = i dx, exact C = exp(-k^4 t) cos(k x); the fitted exponent of
    Eq. (myerr) against N is printed in the caption of Fig. 2 as -2.0162."""
    g = json.load(open(os.path.join(GOLDEN, "paper_convergence.json")))
    k = 2 * math.pi * g["n"] / g["L"]
    T, dt = g["T"], g["dt"]
    steps = int(round(T / dt))
    Ns = [16, 32, 64, 128, 256]
    errs = []
    for N in Ns:
        dx = g["L"] / N
        x = np.arange(N) * dx
        sigma = g["gamma"] * g["D"] * dt / (2 * dx ** 4)
        num = oracle.periodic_steps(N, [sigma], g["amplitude"] * np.cos(k * x + g["phase"]), steps, cn=True)
        exact = g["amplitude"] * math.exp(-g["gamma"] * g["D"] * k ** 4 * T) * np.cos(k * x + g["phase"])
        errs.append(math.sqrt(np.mean((num - exact) ** 2)))
    slope = np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert abs(slope - g["fitted_exponent"]) < 0.03
    assert abs(slope - g["theoretical_exponent"]) < 0.05
