"""Exact rational arithmetic for small periodic systems (test infrastructure only).

This module belongs to the oracle: only tests/, __graft_entry__.smoke() and
bench.py's CPU baseline may import it.  It shares nothing with the CUDA library.

One periodic Crank-Nicolson step of the hyperdiffusion scheme, computed without
rounding: every input double is taken as the rational number it is exactly
(fractions.Fraction(float) is exact), and every operation is done in Python
Fractions, in the order the paper gives:

  * the matrix and right-hand side of the periodic scheme (Sec. 2.2,
    Eq. 1d_hyper_scheme / Eq. matrix_sys): a = e = sigma, b = d = -4 sigma,
    c = 1 + 6 sigma on every row, columns taken modulo n, and
    f_i = -sigma C_{i-2} + 4 sigma C_{i-1} + (1 - 6 sigma) C_i + 4 sigma C_{i+1}
    - sigma C_{i+2};
  * Navon's reduction of the cyclic system (Sec. 2.3): E, the leading
    (n-2) x (n-2) pentadiagonal block; k, its columns n-2, n-1; h^T, the last
    two rows restricted to columns 0..n-3; D, the trailing 2 x 2 block; the
    last two unknowns from Eq. (first_two), S t = f_tail - h^T E^{-1} f-hat with
    S = D - h^T E^{-1} k, and the rest from Eq. (solve),
    x-hat = E^{-1} (f-hat - k t);
  * each E^{-1} by the factorisation and the two substitutions of Sec. 2.4
    (steps 1-14, then the steps for g and for x), the uniform row recurrence
    with out-of-range quantities zero.

A dense Gaussian elimination in Fractions (dense_solve) is the independent
check of the reduction.

Also one step of the 2D Cahn-Hilliard ADI scheme on the no-flux grid, exactly
(adi_step): the delta form's right-hand side mu L(C^3 - C) - sigma L(L C)
(Sec. 2.1, the fourth-order term at the old level), then (I + sigma D4_x) and
(I + sigma D4_y) solved along the rows and the columns by the same Sec. 2.4
recurrences (the no-flux D4 of Sec. 2.2 with its mirrored weights written out),
then dC less its mean (zero in exact arithmetic).  Exact results have no
rounding to compare with: they are the reference that a floating-point step's
error is measured against.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence


def exact(v) -> Fraction:
    """The rational value of a double (or an int / Fraction) exactly."""
    return v if isinstance(v, Fraction) else Fraction(float(v)) if isinstance(v, float) else Fraction(v)


def periodic_hyperdiff_band(n: int, sigma) -> tuple:
    """Eq. (matrix_sys): the same five diagonals on every row of the cyclic matrix."""
    s = exact(sigma)
    return ([s] * n, [-4 * s] * n, [1 + 6 * s] * n, [-4 * s] * n, [s] * n)


def periodic_cn_rhs(sigma, C: Sequence) -> List[Fraction]:
    """Eq. (matrix_sys)'s right-hand side (I - sigma D4) C, indices modulo n."""
    s = exact(sigma)
    c = [exact(v) for v in C]
    n = len(c)
    return [-s * c[(i - 2) % n] + 4 * s * c[(i - 1) % n] + (1 - 6 * s) * c[i] + 4 * s * c[(i + 1) % n]
            - s * c[(i + 2) % n] for i in range(n)]


def factor(a, b, c, d, e):
    """Sec. 2.4, factorisation steps 1-14 (the uniform row recurrence): alpha, beta, gamma, delta, epsilon."""
    m = len(c)
    al, be, ga, de, ep = ([Fraction(0)] * m for _ in range(5))
    for i in range(m):
        ai = a[i] if i >= 2 else 0
        bi = b[i] if i >= 1 else 0
        di = d[i] if i + 1 < m else 0
        ei = e[i] if i + 2 < m else 0
        ep[i] = ai
        be[i] = bi - (ai * ga[i - 2] if i >= 2 else 0)
        al[i] = c[i] - (ai * de[i - 2] if i >= 2 else 0) - (be[i] * ga[i - 1] if i >= 1 else 0)
        if al[i] == 0:
            raise ZeroDivisionError(f"zero pivot at row {i}")
        ga[i] = (di - (be[i] * de[i - 1] if i >= 1 else 0)) / al[i]
        de[i] = ei / al[i]
    return al, be, ga, de, ep


def solve(fac, f) -> List[Fraction]:
    """Sec. 2.4: L g = f (g_i = (f_i - epsilon_i g_{i-2} - beta_i g_{i-1}) / alpha_i), then
    R x = g (x_i = g_i - gamma_i x_{i+1} - delta_i x_{i+2})."""
    al, be, ga, de, ep = fac
    m = len(al)
    g = [Fraction(0)] * m
    for i in range(m):
        v = exact(f[i])
        if i >= 2:
            v -= ep[i] * g[i - 2]
        if i >= 1:
            v -= be[i] * g[i - 1]
        g[i] = v / al[i]
    x = [Fraction(0)] * m
    for i in range(m - 1, -1, -1):
        v = g[i]
        if i + 1 < m:
            v -= ga[i] * x[i + 1]
        if i + 2 < m:
            v -= de[i] * x[i + 2]
        x[i] = v
    return x


def navon_solve(band, f) -> List[Fraction]:
    """Sec. 2.3: the cyclic system A x = f (n >= 5) by Navon's reduction."""
    a, b, c, d, e = ([exact(v) for v in diag] for diag in band)
    n = len(c)
    m = n - 2
    # E: rows and columns 0..m-1; its out-of-range entries are not read by factor()
    fac = factor(a[:m], b[:m], c[:m], d[:m], e[:m])
    # k: rows 0..m-1 in columns n-2, n-1
    k0 = [Fraction(0)] * m
    k1 = [Fraction(0)] * m
    k0[0] += a[0]          # row 0 reaches column (0 - 2) mod n = n-2
    k1[0] += b[0]          # and column n-1
    k1[1] += a[1]          # row 1 reaches column n-1
    k0[m - 2] += e[m - 2]  # row m-2, column m = n-2
    k0[m - 1] += d[m - 1]  # row m-1, column n-2
    k1[m - 1] += e[m - 1]  # row m-1, column n-1
    # h^T: rows n-2, n-1 in columns 0..m-1
    h0 = [Fraction(0)] * m
    h1 = [Fraction(0)] * m
    h0[m - 2] += a[n - 2]
    h0[m - 1] += b[n - 2]
    h0[0] += e[n - 2]      # row n-2 reaches column n mod n = 0
    h1[m - 1] += a[n - 1]
    h1[0] += d[n - 1]
    h1[1] += e[n - 1]
    # D: the trailing 2 x 2 block
    D = [[c[n - 2], d[n - 2]], [b[n - 1], c[n - 1]]]
    fhat = [exact(v) for v in f[:m]]
    q0 = solve(fac, k0)
    q1 = solve(fac, k1)
    y = solve(fac, fhat)
    # Eq. (first_two): (D - h^T E^{-1} k) t = f_tail - h^T E^{-1} f-hat
    S = [[D[0][0] - sum(h0[i] * q0[i] for i in range(m)), D[0][1] - sum(h0[i] * q1[i] for i in range(m))],
         [D[1][0] - sum(h1[i] * q0[i] for i in range(m)), D[1][1] - sum(h1[i] * q1[i] for i in range(m))]]
    r0 = exact(f[n - 2]) - sum(h0[i] * y[i] for i in range(m))
    r1 = exact(f[n - 1]) - sum(h1[i] * y[i] for i in range(m))
    det = S[0][0] * S[1][1] - S[0][1] * S[1][0]
    if det == 0:
        raise ZeroDivisionError("singular 2 x 2 Schur complement")
    t0 = (S[1][1] * r0 - S[0][1] * r1) / det
    t1 = (S[0][0] * r1 - S[1][0] * r0) / det
    # Eq. (solve): E x-hat = f-hat - k t
    xhat = solve(fac, [fhat[i] - k0[i] * t0 - k1[i] * t1 for i in range(m)])
    return xhat + [t0, t1]


def periodic_cn_step(sigma, C: Sequence) -> List[Fraction]:
    """One periodic Crank-Nicolson step (I + sigma D4) C' = (I - sigma D4) C, exactly."""
    return navon_solve(periodic_hyperdiff_band(len(C), sigma), periodic_cn_rhs(sigma, C))


def periodic_matrix(band) -> List[List[Fraction]]:
    """The dense cyclic matrix of a band (columns modulo n)."""
    a, b, c, d, e = ([exact(v) for v in diag] for diag in band)
    n = len(c)
    A = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        for off, diag in ((-2, a), (-1, b), (0, c), (1, d), (2, e)):
            A[i][(i + off) % n] += diag[i]
    return A


def dense_solve(A, f) -> List[Fraction]:
    """Gaussian elimination with row pivoting on a nonzero entry, in Fractions."""
    n = len(A)
    M = [[exact(v) for v in row] + [exact(f[i])] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(col + 1, n):
            if M[r][col] != 0:
                q = M[r][col] / M[col][col]
                M[r] = [x - q * y for x, y in zip(M[r], M[col])]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        x[i] = (M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))) / M[i][i]
    return x


# ----------------------------------------------------------------------------- no-flux grids, the ADI step

def noflux_d4_weights(i: int, n: int) -> List[int]:
    """Sec. 2.2: the centred fourth difference [1, -4, 6, -4, 1] on row i of an n-row cell-centred
    grid with no-flux walls: a column outside 0..n-1 is mirrored about the wall (-1 -> 0, -2 -> 1,
    n -> n-1, n+1 -> n-2, again for very short grids) and its weight added there.  Returns the
    weights of columns i-2 .. i+2 (a weight mirrored outside that window is not possible for n >= 2)."""
    w = [0] * 5
    for k, c in enumerate((1, -4, 6, -4, 1)):
        j = i + k - 2
        while j < 0 or j >= n:
            j = -1 - j if j < 0 else 2 * n - 1 - j
        w[j - i + 2] += c
    return w


def noflux_hyperdiff_band(n: int, sigma) -> tuple:
    """The band (a, b, c, d, e) of I + sigma D4 on the no-flux grid, exactly: row i holds a_i at
    column i-2, ..., e_i at column i+2."""
    s = exact(sigma)
    a, b, c, d, e = ([Fraction(0)] * n for _ in range(5))
    for i in range(n):
        w = noflux_d4_weights(i, n)
        a[i], b[i], c[i], d[i], e[i] = s * w[0], s * w[1], 1 + s * w[2], s * w[3], s * w[4]
    return a, b, c, d, e


def band_apply(band, x) -> List[Fraction]:
    """A x for a band (a, b, c, d, e), exactly."""
    a, b, c, d, e = band
    n = len(c)
    x = [exact(v) for v in x]
    return [sum(coef[i] * x[i + off] for off, coef in ((-2, a), (-1, b), (0, c), (1, d), (2, e)) if 0 <= i + off < n)
            for i in range(n)]


def laplacian_noflux(V) -> List[List[Fraction]]:
    """The five-point Laplacian in grid units with the no-flux mirror (the ghost beyond a wall equals
    the cell next to it), on a list of ny rows of nx values, exactly."""
    ny, nx = len(V), len(V[0])
    v = [[exact(q) for q in row] for row in V]
    out = [[Fraction(0)] * nx for _ in range(ny)]
    for y in range(ny):
        for x in range(nx):
            c0 = v[y][x]
            w = v[y][x - 1] if x > 0 else c0
            ea = v[y][x + 1] if x + 1 < nx else c0
            s = v[y - 1][x] if y > 0 else c0
            nn = v[y + 1][x] if y + 1 < ny else c0
            out[y][x] = (w - 2 * c0 + ea) + (s - 2 * c0 + nn)
    return out


def ch_rhs(C, mu, sigma) -> List[List[Fraction]]:
    """The delta form's right-hand side mu L(C^3 - C) - sigma L(L C) (Sec. 2.1's explicit part of the
    semi-implicit Cahn-Hilliard step with D = 1, the fourth-order term at the old level), exactly."""
    c = [[exact(q) for q in row] for row in C]
    u = [[q * q * q - q for q in row] for row in c]
    lu, llc = laplacian_noflux(u), laplacian_noflux(laplacian_noflux(c))
    m, s = exact(mu), exact(sigma)
    return [[m * lu[y][x] - s * llc[y][x] for x in range(len(c[0]))] for y in range(len(c))]


def adi_delta(rhs, sigma) -> List[List[Fraction]]:
    """dC with (I + sigma D4_x)(I + sigma D4_y) dC = rhs: every grid row solved along x, then every
    column along y, each by the Sec. 2.4 factorisation and substitutions of the shared band."""
    ny, nx = len(rhs), len(rhs[0])
    fx = factor(*noflux_hyperdiff_band(nx, sigma))
    W = [solve(fx, row) for row in rhs]
    fy = factor(*noflux_hyperdiff_band(ny, sigma))
    cols = [solve(fy, [W[y][x] for y in range(ny)]) for x in range(nx)]
    return [[cols[x][y] for x in range(nx)] for y in range(ny)]


def adi_step(C, mu, sigma) -> List[List[Fraction]]:
    """One Douglas ADI step of 2D Cahn-Hilliard in the delta form (the reading of Sec. 4's ADI remark that
    the library and the oracle share): dC from adi_delta of ch_rhs, its mean removed (zero exactly:
    L and D4 have zero column sums), C + dC."""
    dC = adi_delta(ch_rhs(C, mu, sigma), sigma)
    ny, nx = len(dC), len(dC[0])
    mean = sum(sum(row) for row in dC) / (nx * ny)
    return [[exact(C[y][x]) + dC[y][x] - mean for x in range(nx)] for y in range(ny)]
