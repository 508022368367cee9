"""Pins for the oracle's semi-implicit steps with an explicit part: the
Cahn-Hilliard step of Sec. 2.1 (Eq. temporal) and the Crank-Nicolson
hyperdiffusion step of Sec. 2.2 (Eq. 1d_hyper_scheme), on the no-flux and the
periodic grid.  Checked against dense matrices built by hand, exact mass
conservation, closed-form mode amplification factors and fixed points.  No GPU."""
import math

import numpy as np
import pytest

import oracle
import synth


def wrap(j, n, periodic):
    if periodic:
        return j % n
    while j < 0 or j >= n:
        j = -1 - j if j < 0 else 2 * n - 1 - j
    return j


def stencil_matrix(n, weights, periodic):
    """Dense matrix of a centred stencil {offset: weight} with reflected or periodic indices."""
    M = np.zeros((n, n))
    for i in range(n):
        for off, w in weights.items():
            M[i, wrap(i + off, n, periodic)] += w
    return M


def D2(n, periodic):
    return stencil_matrix(n, {-1: 1, 0: -2, 1: 1}, periodic)


def D4(n, periodic):
    return stencil_matrix(n, {-2: 1, -1: -4, 0: 6, 1: -4, 2: 1}, periodic)


def ns_for(periodic):
    return [5, 6, 7, 9, 12] if periodic else [1, 2, 3, 4, 5, 9, 12]


@pytest.mark.parametrize("periodic", [False, True])
def test_explicit_rhs_equals_dense_operators(periodic):
    for n in ns_for(periodic):
        C = synth.uniform(60 + n, 0, n, -1, 1)
        mu, nu = 0.37, 1.9
        ref = C + mu * D2(n, periodic) @ (C ** 3 - C) - nu * D4(n, periodic) @ C
        assert np.allclose(oracle.explicit_rhs(C, mu, nu, periodic), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("periodic", [False, True])
def test_one_step_equals_dense_solve(periodic):
    for n in ns_for(periodic):
        C = synth.uniform(70 + n, 0, n, -1, 1)
        sigma, mu, nu = 3.3, 0.8, 0.4
        f = C + mu * D2(n, periodic) @ (C ** 3 - C) - nu * D4(n, periodic) @ C
        ref = np.linalg.solve(np.eye(n) + sigma * D4(n, periodic), f)
        out = oracle.explicit_steps([n], [sigma], [mu], [nu], C, 1, periodic=periodic)
        assert np.max(np.abs(out - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("periodic", [False, True])
def test_cahn_hilliard_conserves_mass(periodic):
    n, batch = 64, 6
    sig = synth.log_uniform(5, 0, batch, 1e-2, 1e2)
    mu = synth.log_uniform(5, batch, batch, 1e-3, 1.0)
    C = synth.uniform(5, 2 * batch, batch * n, -0.9, 0.9)
    out = oracle.explicit_steps(np.full(batch, n), sig, mu, None, C, 30, periodic=periodic)
    for s in range(batch):
        sl = slice(s * n, (s + 1) * n)
        assert abs(out[sl].sum() - C[sl].sum()) <= 1e-12 * np.abs(C[sl]).sum()


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_cahn_hilliard_linear_growth_factor(periodic, k):
    """Near C = 0, C^3 - C ~ -C: a mode with D2 eigenvalue -p grows per step by (1 + mu p) / (1 + sigma p^2)
    (the amplitude 1e-7 keeps the cubic term below 1e-13 of the mode)."""
    n, sigma, mu, T, amp = 48, 0.9, 0.6, 12, 1e-7
    i = np.arange(n)
    if periodic:
        mode = np.cos(2 * math.pi * k * i / n)
        p = 4 * math.sin(math.pi * k / n) ** 2
    else:
        mode = np.cos(math.pi * k * (i + 0.5) / n)
        p = 4 * math.sin(math.pi * k / (2 * n)) ** 2
    G = (1 + mu * p) / (1 + sigma * p * p)
    out = oracle.explicit_steps([n], [sigma], [mu], None, amp * mode, T, periodic=periodic)
    assert np.max(np.abs(out - amp * G ** T * mode)) <= 1e-9 * amp * G ** T


@pytest.mark.parametrize("periodic", [False, True])
def test_crank_nicolson_mode_amplification(periodic):
    """nu = sigma: the hyperdiffusion Crank-Nicolson step multiplies a D4 eigenmode by (1 - s l)/(1 + s l)."""
    n, s, T, k = 40, 1.7, 25, 3
    i = np.arange(n)
    if periodic:
        mode = np.sin(2 * math.pi * k * i / n)
        lam = 16 * math.sin(math.pi * k / n) ** 4
    else:
        mode = np.cos(math.pi * k * (i + 0.5) / n)
        lam = 16 * math.sin(math.pi * k / (2 * n)) ** 4
    G = (1 - s * lam) / (1 + s * lam)
    out = oracle.explicit_steps([n], [s], None, [s], mode, T, periodic=periodic)
    assert np.max(np.abs(out - G ** T * mode)) <= 1e-13


@pytest.mark.parametrize("periodic", [False, True])
def test_constant_field_is_fixed(periodic):
    n, c = 20, 0.3
    out = oracle.explicit_steps([n], [5.0], [0.7], [0.2], np.full(n, c), 10, periodic=periodic)
    assert np.max(np.abs(out - c)) <= 1e-14


def test_periodic_crank_nicolson_equals_the_navon_driver():
    """The periodic driver with nu = sigma runs the same scheme as the Crank-Nicolson steps of Sec. 2.3."""
    n, batch = 33, 3
    sig = np.array([0.2, 5.0, 80.0])
    C = synth.uniform(21, 0, batch * n, -1, 1)
    a = oracle.explicit_steps(np.full(batch, n), sig, None, sig, C, 7, periodic=True)
    b = oracle.periodic_steps(n, sig, C, 7, cn=True)
    assert np.max(np.abs(a - b)) <= 1e-13
