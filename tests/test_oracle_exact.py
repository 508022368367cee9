"""Pins of the exact periodic Crank-Nicolson step (oracle/exact.py): Navon's reduction
in rational arithmetic equals a dense rational solve of the cyclic matrix exactly;
a constant field is a fixed point; and the FP64 oracle's step lies within the
forward-error bound of its own floating-point evaluation, which is what sets
the periodic tests' bar at the workload's sigma.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import exact as ex

SIGMA_WORKLOAD = 1e-8 / (2 * (1.0 / 512) ** 4)  # sigma_x = dt / (2 dx^4) of the periodic workload, ~343.6


@pytest.mark.parametrize("n", [5, 6, 7, 9])
@pytest.mark.parametrize("sigma", [0.7, SIGMA_WORKLOAD])
def test_navon_reduction_equals_dense_rational_solve(n, sigma):
    band = ex.periodic_hyperdiff_band(n, sigma)
    f = [Fraction(v) for v in synth.uniform(900 + n, 0, n, -1, 1)]
    assert ex.navon_solve(band, f) == ex.dense_solve(ex.periodic_matrix(band), f)


@pytest.mark.parametrize("n", [5, 8, 11])
def test_navon_reduction_general_cyclic_band(n):
    band = synth.random_bands(1, n, seed=950 + n, kind="diagdom")
    f = synth.uniform(960 + n, 0, n, -1, 1)
    x = ex.navon_solve(band, f)
    assert x == ex.dense_solve(ex.periodic_matrix(band), f)
    # and A x = f exactly
    A = ex.periodic_matrix(band)
    assert all(sum(A[i][j] * x[j] for j in range(n)) == Fraction(float(f[i])) for i in range(n))


def test_crank_nicolson_step_fixed_point_and_dense_check():
    n = 7
    assert ex.periodic_cn_step(SIGMA_WORKLOAD, [0.25] * n) == [Fraction(1, 4)] * n
    C = synth.uniform(970, 0, n, -1, 1)
    band = ex.periodic_hyperdiff_band(n, SIGMA_WORKLOAD)
    rhs = ex.periodic_cn_rhs(SIGMA_WORKLOAD, C)
    assert ex.periodic_cn_step(SIGMA_WORKLOAD, C) == ex.dense_solve(ex.periodic_matrix(band), rhs)


def fp64_cn_bound(sigma, C):
    """Forward-error bound of one FP64 Crank-Nicolson step relative to the exact one, per element:
    the right-hand side sums five rounded products of magnitude up to (1 + 16 sigma) max|C| in all
    (gamma_6 (1 + 16 sigma) max|C|, gamma_6 = 6u / (1 - 6u)), and the solve then adds about
    kappa u of its result (kappa ~ 1 + 32 sigma for the cyclic matrix, the solve being backward
    stable); u = 2^-53."""
    u = 2.0 ** -53
    g6 = 6 * u / (1 - 6 * u)
    return g6 * (1 + 16 * sigma) * np.max(np.abs(C)), (1 + 32 * sigma) * u


@pytest.mark.parametrize("n", [64, 128])
def test_fp64_oracle_lies_within_its_forward_error_bound(n):
    """The FP64 oracle's periodic step against the exact step at the workload's sigma: within the
    bound of its own rounding, about 3.7e-12 of max|C'| here -- the periodic tests' bar, explained."""
    C = synth.uniform(980 + n, 0, n, -1, 1)
    xe = np.array([float(v) for v in ex.periodic_cn_step(SIGMA_WORKLOAD, C)])
    xo = oracle.periodic_steps(n, np.array([SIGMA_WORKLOAD]), C, 1, cn=True, shared=True)
    rhs_bound, kappa_u = fp64_cn_bound(SIGMA_WORKLOAD, C)
    bound = rhs_bound + kappa_u * np.max(np.abs(xe))
    err = np.max(np.abs(xo - xe))
    print(f"n={n}: FP64 oracle vs exact {err / np.max(np.abs(xe)):.2e} of max|C'|, bound {bound / np.max(np.abs(xe)):.2e}")
    assert err <= bound


# ----------------------------------------------------------------------------- the exact ADI step

def _grid(ny, nx, seed):
    return synth.uniform(seed, 0, nx * ny, -0.1, 0.1).reshape(ny, nx)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 13])
@pytest.mark.parametrize("sigma", [0.5, 0.25, 2.0])
def test_noflux_band_equals_the_oracles(n, sigma):
    """The exact no-flux band (its mirrored D4 weights written out here) equals the C oracle's band
    entry by entry where sigma times the weights is exact in FP64 (a power of two)."""
    e = ex.noflux_hyperdiff_band(n, sigma)
    o = oracle.band_hyperdiff(n, sigma)
    inside = [lambda i: i >= 2, lambda i: i >= 1, lambda i: True, lambda i: i + 1 < n, lambda i: i + 2 < n]
    for k in range(5):
        for i in range(n):
            if inside[k](i):
                assert Fraction(float(o[k][i])) == e[k][i], (k, i)
    # D4 reflected is symmetric with zero row sums, so I + sigma D4 has unit row and column sums
    for i in range(n):
        row = [e[0][i], e[1][i], e[2][i], e[3][i], e[4][i]]
        assert sum(c for off, c in zip(range(-2, 3), row) if 0 <= i + off < n) == 1


@pytest.mark.parametrize("ny,nx,sigma", [(5, 7, 0.7), (9, 6, 343.6), (10, 12, 1.76e5)])
def test_exact_adi_delta_solves_both_factors_and_keeps_the_mass(ny, nx, sigma):
    """(I + sigma D4_x)(I + sigma D4_y) dC = rhs holds exactly for the exact dC, whose sum is exactly
    zero (L has zero column sums and both factors unit ones), so the mean the step removes is zero
    and the step keeps sum C exactly."""
    C = _grid(ny, nx, 11)
    mu = 0.41
    rhs = ex.ch_rhs(C.tolist(), mu, sigma)
    assert sum(sum(r) for r in rhs) == 0
    dC = ex.adi_delta(rhs, sigma)
    bx, by = ex.noflux_hyperdiff_band(nx, sigma), ex.noflux_hyperdiff_band(ny, sigma)
    Y = [ex.band_apply(by, [dC[y][x] for y in range(ny)]) for x in range(nx)]  # y factor, per column
    back = [ex.band_apply(bx, [Y[x][y] for x in range(nx)]) for y in range(ny)]  # then the x factor
    assert back == rhs
    assert sum(sum(r) for r in dC) == 0
    C1 = ex.adi_step(C.tolist(), mu, sigma)
    assert sum(sum(r) for r in C1) == sum(ex.exact(v) for v in C.ravel())


@pytest.mark.parametrize("ny,nx,dt,dx,bar", [(10, 12, 1e-4, 1 / 64, 1e-13), (20, 24, 1e-6, 1 / 2048, 2e-9)])
def test_fp64_oracle_adi_step_near_the_exact_step(ny, nx, dt, dx, bar):
    """The FP64 oracle's step against the exact step on the same doubles (relative to max|dC|): at
    sigma = 16.8 to within rounding; at the workload's sigma = 1.76e5, where the factors'
    condition is ~3e6, within that condition times FP64 rounding (measured 3e-10)."""
    C = _grid(ny, nx, 12)
    gamma = 0.01
    mu, sigma = dt / (dx * dx), gamma * dt / (dx * dx * dx * dx)
    E = np.array([[float(v) for v in row] for row in ex.adi_step(C.tolist(), mu, sigma)])
    O = oracle.adi_step(C, gamma, dt, dx)
    assert np.max(np.abs(O - E)) <= bar * np.max(np.abs(E - C))
