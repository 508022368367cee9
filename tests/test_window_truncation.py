"""The windowed solve's truncation (the reading behind PENT_OPT_WINDOW_WARPS and
PENT_OPT_WINDOW_ROWS), checked on the CPU in plain FP64 numpy, independently of the CUDA path.

A window runs the two substitutions (Sec. 2.4) of a long hyperdiffusion system over its own rows
only, entering with a zero state where it cuts the system (and, away from the walls, with the
interior factors from its first row on), and keeps the rows at least O from a cut.  O is the fewest
multiple of 8 rows at which both 8-row interior chunk maps (forward on (g_{i-2}, g_{i-1}), back on
(x_{i+1}, x_{i+2})) have every entry at most 2^-56.  The rows kept must equal the whole system's
solution to FP64 rounding, for every sigma that windows are used for; the kernels compute O the
same way (in FP64, from the interior factors), and their own tests hold the windowed GPU solves
to the oracle.  The last test pins the form of the forward step that the FP64 system windows
take (the coefficients beta/alpha and sigma/alpha formed once) against the oracle's solve."""
import numpy as np
import pytest

import oracle
import synth

TOL_WIN = 2.0 ** -56


def interior_factors(n, sigma):
    """1/alpha and beta of an interior row of I + sigma D4 (Sec. 2.4's recurrences, FP64)."""
    a, b, c, d, e = oracle.band_hyperdiff(n, sigma)
    al, be, ga, de = (np.zeros(n) for _ in range(4))
    for i in range(n):
        ai = a[i] if i >= 2 else 0.0
        bi = b[i] if i >= 1 else 0.0
        be[i] = bi - (ai * ga[i - 2] if i >= 2 else 0.0)
        al[i] = c[i] - (ai * de[i - 2] if i >= 2 else 0.0) - (be[i] * ga[i - 1] if i >= 1 else 0.0)
        ga[i] = ((d[i] if i + 1 < n else 0.0) - (be[i] * de[i - 1] if i >= 1 else 0.0)) / al[i]
        de[i] = (e[i] if i + 2 < n else 0.0) / al[i]
    m = n // 2
    return 1.0 / al[m], be[m]


def overlap_rows(ia, bi, sigma, L=8, kmax=64):
    """O: the fewest k L with max |entry| of M_f^k and M_b^k at most 2^-56 (None past kmax)."""
    Rf = np.array([[0.0, 1.0], [-ia * sigma, -ia * bi]])
    Rb = np.array([[-ia * bi, -ia * sigma], [1.0, 0.0]])
    Mf = np.linalg.matrix_power(Rf, L)
    Mb = np.linalg.matrix_power(Rb, L)
    P, Q = Mf.copy(), Mb.copy()
    for k in range(1, kmax + 1):
        if max(np.abs(P).max(), np.abs(Q).max()) <= TOL_WIN:
            return k * L
        P, Q = Mf @ P, Mb @ Q
    return None


def window_solve(f, ia, bi, sigma):
    """Both substitutions over a window with the interior factors throughout, zero states at both
    cuts."""
    m = len(f)
    g = np.zeros(m)
    p2 = p1 = 0.0
    for i in range(m):
        gi = ia * (f[i] - bi * p1 - sigma * p2)
        g[i] = gi
        p2, p1 = p1, gi
    x = np.zeros(m)
    s1 = s2 = 0.0
    for i in range(m - 1, -1, -1):
        xi = g[i] - ia * (bi * s1 + sigma * s2)
        x[i] = xi
        s2, s1 = s1, xi
    return x


@pytest.mark.parametrize("sigma", [1e-3, 1e-2, 0.1, 1.0, 3.0, 10.0, 30.0])
def test_kept_rows_equal_the_whole_solve(sigma):
    n = 4000
    ia, bi = interior_factors(n, sigma)
    O = overlap_rows(ia, bi, sigma)
    assert O is not None and O % 8 == 0
    R = 1024 if O <= 128 else 2048  # the window whose overlap room (R / 8) takes this sigma
    assert O <= R // 8
    f = synth.uniform(501, 0, n, -1.0, 1.0)
    fac, bad = oracle.factor(oracle.band_hyperdiff(n, sigma))
    assert bad == -1
    x = oracle.solve(fac, f)
    for w0 in (1000, 1960):  # windows well inside the system
        xw = window_solve(f[w0:w0 + R], ia, bi, sigma)
        kept = slice(O, R - O)
        err = np.max(np.abs(xw[kept] - x[w0:w0 + R][kept]))
        assert err <= 1e-14 * np.max(np.abs(x)), (sigma, O, err)
    # and a shorter overlap is not enough where the decay is slow (the criterion is not loose)
    if sigma >= 1.0:
        xw = window_solve(f[1000:1000 + R], ia, bi, sigma)
        short = slice(O // 4, R - O // 4)
        assert np.max(np.abs(xw[short] - x[1000:1000 + R][short])) > 1e-12 * np.max(np.abs(x))


def test_overlap_grows_with_sigma():
    """Slower decay, longer overlap: about 16 rows at sigma = 0.01, 96 at 10, beyond the 1024-row
    windows' room (128) near sigma = 100."""
    Os = []
    for sigma in (1e-2, 0.1, 1.0, 10.0, 100.0):
        ia, bi = interior_factors(2000, sigma)
        Os.append(overlap_rows(ia, bi, sigma))
    assert all(a is not None for a in Os[:4])
    assert Os[:4] == sorted(Os[:4])
    assert Os[0] <= 24 and 80 <= Os[3] <= 104
    assert Os[4] is None or Os[4] > 128


@pytest.mark.parametrize("sigma", [1e-3, 0.1, 1.0, 10.0, 30.0])
def test_forward_step_with_its_coefficients_formed_once(sigma):
    """The FP64 system windows' forward step, g_i = (1/alpha_i) f_i - (beta_i/alpha_i) g_{i-1}
    - (sigma/alpha_i) g_{i-2}, with beta_i/alpha_i and sigma/alpha_i formed once per row as
    products with the stored 1/alpha_i, followed by the back substitution, agrees with the oracle's
    solve (Sec. 2.4's division form) to FP64 rounding; and the hyperdiffusion band's epsilon_i
    (= a_i) is exactly sigma on every row from 2 on, which every hyperdiffusion walk takes instead
    of a stored epsilon."""
    n = 3001
    fac, bad = oracle.factor(oracle.band_hyperdiff(n, sigma))
    assert bad == -1
    al, be, ga, de, ep = fac
    assert np.all(ep[2:] == sigma)
    f = synth.uniform(502, 0, n, -1.0, 1.0)
    ia = 1.0 / al
    iab, ias = ia * be, ia * sigma
    g = np.zeros(n)
    g1 = g2 = 0.0
    for i in range(n):
        g[i] = ia[i] * f[i] - ias[i] * g2 - iab[i] * g1
        g2, g1 = g1, g[i]
    x = np.zeros(n)
    x1 = x2 = 0.0
    for i in range(n - 1, -1, -1):
        x[i] = g[i] - ga[i] * x1 - de[i] * x2
        x2, x1 = x1, x[i]
    ref = oracle.solve(fac, f)
    assert np.max(np.abs(x - ref)) <= 1e-14 * np.max(np.abs(ref))
