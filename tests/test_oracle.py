"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- exact rational arithmetic, a dense library solve, closed forms,
invariants, brute-force stencils and values the paper prints.  No GPU needed."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- independent helpers

def dense(band):
    """Dense matrix with row i = a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1} + e_i x_{i+2}."""
    a, b, c, d, e = band
    n = len(c)
    A = np.zeros((n, n))
    for i in range(n):
        for off, v in ((-2, a), (-1, b), (0, c), (1, d), (2, e)):
            j = i + off
            if 0 <= j < n:
                A[i, j] = v[i]
    return A


def crout_exact(A):
    """Exact A = L R (L lower, R unit upper) in rational arithmetic, no pivoting."""
    n = len(A)
    L = [[Fraction(0)] * n for _ in range(n)]
    R = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for j in range(n):
        for i in range(j, n):
            L[i][j] = A[i][j] - sum((L[i][k] * R[k][j] for k in range(j)), Fraction(0))
        for i in range(j + 1, n):
            R[j][i] = (A[j][i] - sum((L[j][k] * R[k][i] for k in range(j)), Fraction(0))) / L[j][j]
    return L, R


def mirror(j, n):
    """Cell-centred even reflection of index j into 0..n-1 (ghost C_{-1}=C_0, C_{-2}=C_1, ...)."""
    while j < 0 or j >= n:
        j = -1 - j if j < 0 else 2 * n - 1 - j
    return j


def d4_by_reflection(n):
    D = np.zeros((n, n))
    for i in range(n):
        for off, w in ((-2, 1), (-1, -4), (0, 6), (1, -4), (2, 1)):
            D[i, mirror(i + off, n)] += w
    return D


def lap_by_reflection(v):
    ny, nx = v.shape
    out = np.zeros_like(v)
    for y in range(ny):
        for x in range(nx):
            s = -4.0 * v[y, x]
            s += v[y, mirror(x - 1, nx)] + v[y, mirror(x + 1, nx)]
            s += v[mirror(y - 1, ny), x] + v[mirror(y + 1, ny), x]
            out[y, x] = s
    return out


def rel_err(x, ref):
    return np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300)


def cosmode(n, k):
    return np.cos(np.pi * k * (np.arange(n) + 0.5) / n)


def lam_d4(n, k):
    """Eigenvalue of the no-flux D4 on the cosine mode k: (4 sin^2(pi k / 2n))^2."""
    return 16.0 * math.sin(math.pi * k / (2 * n)) ** 4


# ----------------------------------------------------------------------------- factorisation (Sec. 2.4)

@pytest.mark.parametrize("n", list(range(1, 9)))
def test_factor_equals_exact_rational_lu(n):
    rng = np.random.default_rng(100 + n)
    ints = rng.integers(-3, 4, size=(4, n)).astype(float)
    a, b, d, e = ints
    c = 1.0 + np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e) + rng.integers(0, 3, size=n)
    band = (a, b, c, d, e)
    A = dense(band)
    L, R = crout_exact([[Fraction(int(v)) for v in row] for row in A])
    (al, be, ga, de, ep), bad = oracle.factor(band)
    assert bad == -1
    for i in range(n):
        assert al[i] == pytest.approx(float(L[i][i]), rel=1e-14, abs=1e-14)
        if i >= 1:
            assert be[i] == pytest.approx(float(L[i][i - 1]), rel=1e-14, abs=1e-14)
        if i >= 2:
            assert ep[i] == pytest.approx(float(L[i][i - 2]), rel=1e-14, abs=1e-14)
        if i + 1 < n:
            assert ga[i] == pytest.approx(float(R[i][i + 1]), rel=1e-14, abs=1e-14)
        if i + 2 < n:
            assert de[i] == pytest.approx(float(R[i][i + 2]), rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("kind", ["diagdom", "spd"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 16, 33])
def test_L_times_R_equals_A(kind, n):
    band = synth.random_bands(1, n, seed=7 + n, kind=kind)
    (al, be, ga, de, ep), bad = oracle.factor(band)
    assert bad == -1
    L, R = np.zeros((n, n)), np.eye(n)
    for i in range(n):
        L[i, i] = al[i]
        if i >= 1:
            L[i, i - 1] = be[i]
        if i >= 2:
            L[i, i - 2] = ep[i]
        if i + 1 < n:
            R[i, i + 1] = ga[i]
        if i + 2 < n:
            R[i, i + 2] = de[i]
    A = dense(band)
    assert np.max(np.abs(L @ R - A)) <= 1e-14 * np.max(np.abs(A))


@pytest.mark.parametrize("kind", ["diagdom", "spd"])
@pytest.mark.parametrize("n", list(range(1, 17)) + [100])
def test_solve_matches_dense_gaussian_elimination(kind, n):
    band = synth.random_bands(1, n, seed=31 + n, kind=kind)
    f = synth.uniform(99, 0, n, -1.0, 1.0)
    fac, bad = oracle.factor(band)
    assert bad == -1
    x = oracle.solve(fac, f)
    ref = np.linalg.solve(dense(band), f)  # LAPACK gesv: partial pivoting
    assert rel_err(x, ref) <= 1e-13


def test_residual_bound_large_n():
    n = 4000
    band = synth.random_bands(1, n, seed=5, kind="diagdom")
    f = synth.uniform(6, 0, n, -1.0, 1.0)
    fac, _ = oracle.factor(band)
    x = oracle.solve(fac, f)
    r = f - oracle.matvec(band, x)
    normA = np.max(np.sum(np.abs(np.stack(band)), axis=0))
    assert np.max(np.abs(r)) <= 10 * 5 * np.finfo(float).eps * normA * np.max(np.abs(x))


def _band_with_zero_pivot(n, row):
    """Rows before `row` are diagonal (no coupling forward), and c_row = 0, so
    alpha_row = c_row - a_row delta_{row-2} - beta_row gamma_{row-1} = 0 exactly."""
    a, b, c, d, e = (np.full(n, v) for v in (0.1, 0.2, 3.0, 0.2, 0.1))
    d[:row] = 0.0
    e[:row] = 0.0
    c[row] = 0.0
    return a, b, c, d, e


def test_zero_pivot_reported():
    assert oracle.factor(_band_with_zero_pivot(6, 0))[1] == 0
    assert oracle.factor(_band_with_zero_pivot(6, 3))[1] == 3
    nsys = np.array([4, 6, 5, 6])
    bands = [synth.random_bands(1, 4, seed=1, kind="diagdom"), _band_with_zero_pivot(6, 3),
             synth.random_bands(1, 5, seed=2, kind="diagdom"), _band_with_zero_pivot(6, 1)]
    cat = tuple(np.concatenate([bb[k] for bb in bands]) for k in range(5))
    _, bad_sys, bad_row = oracle.factor_batch(nsys, cat, nthreads=2)
    assert (bad_sys, bad_row) == (1, 3)


def test_batch_drivers_match_single_system_calls():
    nsys = np.array([1, 2, 3, 5, 17, 64, 3])
    bands = [synth.random_bands(1, int(m), seed=int(m) + 1000, kind="diagdom") for m in nsys]
    cat = tuple(np.concatenate([bb[k] for bb in bands]) for k in range(5))
    f = synth.uniform(3, 0, int(nsys.sum()), -1, 1)
    fac, bad, _ = oracle.factor_batch(nsys, cat, nthreads=3)
    assert bad == -1
    x = oracle.solve_batch(nsys, fac, f, nthreads=3)
    off = oracle.offsets(nsys)
    for s, bb in enumerate(bands):
        o0, o1 = off[s], off[s + 1]
        ref = np.linalg.solve(dense(bb), f[o0:o1])
        assert rel_err(x[o0:o1], ref) <= 1e-13


# ----------------------------------------------------------------------------- adjoint

def test_transpose_band_is_transpose():
    band = synth.random_bands(1, 9, seed=2, kind="diagdom")
    assert np.array_equal(dense(oracle.transpose_band(band)), dense(band).T)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 50])
def test_adjoint_dot_product_identity(n):
    nsys = np.array([n, n + 3])
    bands = [synth.random_bands(1, int(m), seed=int(m) + 77, kind="diagdom") for m in nsys]
    cat = tuple(np.concatenate([bb[k] for bb in bands]) for k in range(5))
    u = synth.uniform(11, 0, int(nsys.sum()), -1, 1)
    v = synth.uniform(12, 0, int(nsys.sum()), -1, 1)
    fac, _, _ = oracle.factor_batch(nsys, cat)
    Ainv_u = oracle.solve_batch(nsys, fac, u)
    AinvT_v = oracle.adjoint_solve_batch(nsys, cat, v)
    off = oracle.offsets(nsys)
    for s in range(2):
        sl = slice(off[s], off[s + 1])
        lhs, rhs = np.dot(Ainv_u[sl], v[sl]), np.dot(u[sl], AinvT_v[sl])
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(u[sl]) * np.linalg.norm(v[sl]))
        ref = np.linalg.solve(dense(bands[s]).T, v[sl])
        assert rel_err(AinvT_v[sl], ref) <= 1e-13


# ----------------------------------------------------------------------------- hyperdiffusion band (Sec. 2.2-2.3)

@pytest.mark.parametrize("n", list(range(1, 13)))
def test_d4_band_equals_reflected_stencil(n):
    assert np.array_equal(dense(oracle.band_d4(n)), d4_by_reflection(n))


def test_d4_interior_is_the_paper_stencil():
    a, b, c, d, e = oracle.band_d4(10)
    assert list(a[2:8]) == [1] * 6 and list(b[2:8]) == [-4] * 6 and list(c[2:8]) == [6] * 6
    assert list(d[2:8]) == [-4] * 6 and list(e[2:8]) == [1] * 6
    # no-flux rows 0 and 1 (and their mirror images)
    assert (c[0], d[0], e[0]) == (2, -3, 1) and (b[1], c[1], d[1], e[1]) == (-3, 6, -4, 1)
    assert (c[9], b[9], a[9]) == (2, -3, 1) and (d[8], c[8], b[8], a[8]) == (-3, 6, -4, 1)


@pytest.mark.parametrize("n,sigma", [(1, 0.5), (2, 3.0), (5, 0.5), (64, 0.5), (256, 10.0), (1000, 1e-3)])
def test_hyperdiff_band_spectrum_symmetry_and_mass(n, sigma):
    band = oracle.band_hyperdiff(n, sigma)
    A = dense(band)
    assert np.array_equal(A, A.T)
    assert np.allclose(A.sum(axis=0), 1.0, rtol=0, atol=1e-12 * (1 + 16 * sigma))
    for k in sorted({0, 1, 2, n // 3, n - 1}):
        v = cosmode(n, k)
        lam = 1.0 + sigma * lam_d4(n, k)
        assert np.max(np.abs(A @ v - lam * v)) <= 1e-12 * lam


@pytest.mark.parametrize("k", [0, 1, 2, 5, 31])
def test_hyperdiff_steps_cosine_amplification(k):
    n, sigma, steps = 64, 0.5, 100
    v = cosmode(n, k)
    out = oracle.hyperdiff_steps([n], [sigma], v, steps)
    G = 1.0 / (1.0 + sigma * lam_d4(n, k))
    ref = G ** steps * v
    # relative 1e-13 on the mode, plus an absolute floor for the rounding of the initial
    # cosine values, whose components in slowly decaying modes survive the 100 steps
    assert np.max(np.abs(out - ref)) <= 1e-13 * G ** steps + 1e-14


def test_hyperdiff_mass_conserved():
    w = synth.hyperdiff_parametric(batch=8, n=200, steps=100)
    out = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, w.steps)
    off = w.offsets
    for s in range(w.batch):
        m0 = w.field0[off[s]:off[s + 1]].sum()
        m1 = out[off[s]:off[s + 1]].sum()
        assert abs(m1 - m0) <= 1e-13 * np.abs(w.field0[off[s]:off[s + 1]]).sum()


def test_convergence_exponent_matches_paper_fig2():
    """No-flux analogue of the paper's validation (Sec. 2.5): C0 = cos(k x), k = 2 pi n / L,
    exact C = exp(-k^4 t) cos(k x), error of Eq. (myerr) at T, fitted against N."""
    g = json.load(open(os.path.join(GOLDEN, "paper_convergence.json")))
    k = 2 * math.pi * g["n"] / g["L"]
    T, dt = g["T"], g["dt"]
    steps = int(round(T / dt))
    Ns = [16, 32, 64, 128]
    errs = []
    for N in Ns:
        dx = g["L"] / N
        x = (np.arange(N) + 0.5) * dx
        c0 = g["amplitude"] * np.cos(k * x + g["phase"])
        sigma = g["gamma"] * g["D"] * dt / dx ** 4
        num = oracle.hyperdiff_steps([N], [sigma], c0, steps)
        exact = g["amplitude"] * math.exp(-g["gamma"] * g["D"] * k ** 4 * T) * np.cos(k * x + g["phase"])
        errs.append(math.sqrt(np.mean((num - exact) ** 2)))
    slope = np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert abs(slope - g["theoretical_exponent"]) < 0.1
    assert abs(slope - g["fitted_exponent"]) < 0.1


# ----------------------------------------------------------------------------- 2D ADI step (Sec. 4 reading)

def test_laplacian_equals_reflected_stencil():
    v = synth.uniform(4, 0, 35, -1, 1).reshape(5, 7)
    assert np.allclose(oracle.laplacian_noflux(v), lap_by_reflection(v), rtol=0, atol=1e-15)


def test_ch_rhs_brute_force():
    C = synth.uniform(8, 0, 6 * 9, -0.1, 0.1).reshape(6, 9)
    mu, sigma = 4.2, 1.7e5
    ref = mu * lap_by_reflection(C ** 3 - C) - sigma * lap_by_reflection(lap_by_reflection(C))
    out = oracle.ch_rhs(C, mu, sigma)
    assert rel_err(out, ref) <= 1e-14


def _mode2d(nx, ny, kx, ky):
    return np.outer(cosmode(ny, ky), cosmode(nx, kx))


@pytest.mark.parametrize("kx,ky,sigma", [(1, 2, 0.3), (5, 0, 10.0), (7, 11, 1.76e5), (0, 0, 2.0)])
def test_adi_solve_separable_mode(kx, ky, sigma):
    nx, ny = 24, 20
    rhs = _mode2d(nx, ny, kx, ky)
    out = oracle.adi_solve(rhs, sigma)
    p2, q2 = lam_d4(nx, kx), lam_d4(ny, ky)
    ref = rhs / ((1 + sigma * p2) * (1 + sigma * q2))
    # relative 1e-12 on the mode, plus u * ||A^-1|| * ||rhs|| (||A^-1|| <= 1 here) for the
    # rounding of the input mode, which leaves components in the weakly damped modes
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref)) + 1e-15 * np.max(np.abs(rhs))


@pytest.mark.parametrize("kx,ky,sigma", [(1, 2, 0.3), (3, 4, 50.0), (10, 9, 1.76e5)])
def test_adi_linear_amplification_factor(kx, ky, sigma):
    nx, ny = 16, 24
    C = _mode2d(nx, ny, kx, ky)
    out = oracle.adi_step_ms(C, 0.0, sigma)          # nonlinear term off (mu = 0)
    p = 4 * math.sin(math.pi * kx / (2 * nx)) ** 2
    q = 4 * math.sin(math.pi * ky / (2 * ny)) ** 2
    G = 1 - sigma * (p + q) ** 2 / ((1 + sigma * p * p) * (1 + sigma * q * q))
    # 1e-12 relative, plus the rounding of the dominant right-hand side term sigma L(L C)
    # carried through (I + sigma D4_x)^-1 (I + sigma D4_y)^-1, whose norm is at most 1
    u = np.finfo(float).eps
    bound = 1e-12 * np.max(np.abs(G * C)) + u * sigma * (p + q) ** 2 * np.max(np.abs(C))
    assert np.max(np.abs(out - G * C)) <= bound


def test_adi_mass_conserved_config3_parameters():
    w = synth.ch_adi(nx=48, ny=40, steps=20)
    dx = 1.0 / 2048                      # the full-size grid spacing: sigma ~ 1.76e5, mu ~ 4.19
    C = w.field0.copy()
    m0, scale = C.sum(), np.abs(w.field0).sum()
    for _ in range(w.steps):
        C = oracle.adi_step(C, w.gamma, w.dt, dx)
    assert abs(C.sum() - m0) <= 1e-12 * scale


def test_adi_constant_in_y_reduces_to_1d_delta_form():
    nx, ny, mu, sigma = 32, 6, 3.0, 40.0
    v = 0.1 * cosmode(nx, 3) + 0.05 * cosmode(nx, 1)
    C = np.tile(v, (ny, 1))
    out = oracle.adi_step_ms(C, mu, sigma)
    D2 = lap_by_reflection(v[None, :])[0]          # y-part vanishes for a y-constant row
    u = v ** 3 - v
    rhs = mu * lap_by_reflection(u[None, :])[0] - sigma * lap_by_reflection(D2[None, :])[0]
    fac, _ = oracle.factor(oracle.band_hyperdiff(nx, sigma))
    dC = oracle.solve(fac, rhs)
    ref = v + (dC - dC.mean())
    for y in range(ny):
        assert rel_err(out[y], ref) <= 1e-13


# ----------------------------------------------------------------------------- loss / gradient by the adjoint

def _loss_forward(sigma, c0, target, T):
    batch, n = c0.shape
    x = oracle.hyperdiff_steps(np.full(batch, n), sigma, c0.reshape(-1), T).reshape(batch, n)
    return float(np.sum((x - target) ** 2))


def test_loss_gradient_central_differences():
    w = synth.adjoint_batch(batch=3, n=32, steps=6)
    c0 = w.field0.reshape(3, 32)
    target = oracle.hyperdiff_steps(w.n, w.sigma * 1.01, w.field0, w.steps).reshape(3, 32)
    loss, gc, gs = oracle.hyperdiff_loss_grad(w.sigma, w.steps, c0, target)
    assert loss == pytest.approx(_loss_forward(w.sigma, c0, target, w.steps), rel=1e-13)
    h = 1e-6
    for s in range(3):
        sp, sm = w.sigma.copy(), w.sigma.copy()
        sp[s] += h
        sm[s] -= h
        fd = (_loss_forward(sp, c0, target, w.steps) - _loss_forward(sm, c0, target, w.steps)) / (2 * h)
        assert gs[s] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, loss))
    for (s, i) in [(0, 0), (1, 17), (2, 31), (2, 5)]:
        cp, cm = c0.copy(), c0.copy()
        cp[s, i] += h
        cm[s, i] -= h
        fd = (_loss_forward(w.sigma, cp, target, w.steps) - _loss_forward(w.sigma, cm, target, w.steps)) / (2 * h)
        assert gc[s, i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_loss_gradient_single_mode_closed_form():
    n, k, T, sigma = 40, 3, 7, 0.8
    A0, B0 = 1.3, 0.4
    v = cosmode(n, k)
    c0, target = A0 * v, B0 * v
    loss, gc, gs = oracle.hyperdiff_loss_grad(np.array([sigma]), T, c0[None, :], target[None, :])
    lam = lam_d4(n, k)
    G = 1 / (1 + sigma * lam)
    vv = np.dot(v, v)
    assert loss == pytest.approx((A0 * G ** T - B0) ** 2 * vv, rel=1e-13)
    dL_dsigma = 2 * (A0 * G ** T - B0) * vv * A0 * T * G ** (T - 1) * (-lam * G * G)
    assert gs[0] == pytest.approx(dL_dsigma, rel=1e-12)
    assert rel_err(gc[0], 2 * (A0 * G ** T - B0) * G ** T * v) <= 1e-12


def test_vjp_equals_loss_gradient_with_its_cotangent():
    w = synth.adjoint_batch(batch=3, n=40, steps=5)
    c0 = w.field0.reshape(3, 40)
    target = oracle.hyperdiff_steps(w.n, w.sigma * 1.01, w.field0, w.steps).reshape(3, 40)
    _, gc, gs = oracle.hyperdiff_loss_grad(w.sigma, w.steps, c0, target)
    xT = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, w.steps).reshape(3, 40)
    vc, vs = oracle.hyperdiff_vjp(w.sigma, w.steps, c0, 2.0 * (xT - target))
    assert np.array_equal(vc, gc) and np.array_equal(vs, gs)
