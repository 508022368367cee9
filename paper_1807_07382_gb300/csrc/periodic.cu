// Periodic (cyclic) pentadiagonal systems: Navon's reduction (Sec. 2.3).
//
// A cyclic matrix A (Eq. matrix_sys1: rows wrap around, so the first two rows
// reach the last two columns and the last two rows the first two) is split as
//   [ E    k ] [X]   [f-hat ]
//   [ h^T  D ] [t] = [f_tail]      (m = n - 2 rows in E, t = (x_{n-2}, x_{n-1}))
// with E pentadiagonal.  Eq. (first_two) gives t = S^{-1} (f_tail - h^T E^{-1} f-hat),
// S = D - h^T E^{-1} k, and Eq. (solve) gives X = E^{-1} (f-hat - k t).  As the
// paper recommends, everything that depends on the matrix only is formed once,
// at factorisation time (k_factor_periodic):
//   * the factors of E (Sec. 2.4), as 1/alpha, beta/alpha, epsilon/alpha and gamma, delta;
//   * Z = E^{-T} h (two columns), so h^T E^{-1} f-hat = Z^T f-hat is a dot product
//     that the forward sweep accumulates while it reads f-hat;
//   * W = L^{-1} k (two columns), so that after t is known the back sweep solves
//     R X = g - W t, i.e. subtracts W t from g on the fly;
//   * S^{-1} (2 x 2).
// A solve is therefore still one forward and one back sweep per system (one
// thread per system, as in the paper's Sec. 2.6), reading f once and writing x
// once.  The right-hand side of a time step can be assembled inside the forward
// sweep from the old field (k_solve_periodic<.., true>): the Crank-Nicolson
// right-hand side of Eq. (matrix_sys) or the explicit Cahn-Hilliard term of
// Eq. (temporal), on the periodic grid.
//
// Layout: every per-row quantity of E is stored row-interleaved, rec[r * S + s]
// with S systems (the paper's interleaved layout, Sec. 2.6), or rec[r] for a
// matrix shared by the whole batch; the forward scratch g is interleaved too.
// f and x are in the caller's system-major layout.
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace pent {
namespace {

__device__ __forceinline__ void report_bad(unsigned long long* info, int64_t s, int64_t r) {
  atomicMin(info, ((unsigned long long)s << 32) | (unsigned long long)(uint32_t)r);
}

// Band of row i (0 <= i < n) of the cyclic system s: coefficients of
// x_{i-2}, x_{i-1}, x_i, x_{i+1}, x_{i+2} (indices modulo n).  From sigma:
// the periodic hyperdiffusion matrix of Eq. (matrix_sys).
__device__ __forceinline__ void cyc_band(const PerArgs& A, int64_t s, int64_t i, const double* a, const double* b,
                                         const double* c, const double* d, const double* e, const double* sigma,
                                         double& ar, double& br, double& cr, double& dr, double& er) {
  if (sigma) {
    const double sg = sigma[A.shared ? 0 : s];
    ar = sg;
    br = -4.0 * sg;
    cr = 1.0 + 6.0 * sg;
    dr = -4.0 * sg;
    er = sg;
  } else {
    const int64_t o = (A.shared ? 0 : s) * A.n + i;
    ar = a[o];
    br = b[o];
    cr = c[o];
    dr = d[o];
    er = e[o];
  }
}

// One thread per matrix: factor E (Sec. 2.4 steps, generic row step with
// out-of-range terms zero), then W = L^{-1} k, Z = E^{-T} h and S^{-1}.
__global__ void k_factor_periodic(PerArgs A, const double* __restrict__ a, const double* __restrict__ b,
                                  const double* __restrict__ c, const double* __restrict__ d,
                                  const double* __restrict__ e, const double* __restrict__ sigma) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t S = A.shared ? 1 : A.batch;
  if (s >= S) return;
  const int64_t n = A.n, m = A.m;
  auto at = [&](double* p, int64_t r) -> double& { return p[r * S + s]; };
  // ---- factor E ----
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;
  bool failed = false;
  for (int64_t r = 0; r < m; ++r) {
    double ar, br, cr, dr, er;
    cyc_band(A, s, r, a, b, c, d, e, sigma, ar, br, cr, dr, er);
    if (r < 2) ar = 0.0;       // column r - 2 < 0 wraps into k
    if (r < 1) br = 0.0;
    if (r + 1 >= m) dr = 0.0;  // columns >= m belong to k
    if (r + 2 >= m) er = 0.0;
    const double beta = br - ar * gam2;
    const double alpha = cr - ar * del2 - beta * gam1;
    if (!(alpha != 0.0) || !isfinite(alpha)) {
      report_bad(A.info, s, r);
      failed = true;
      break;
    }
    const double gamma = (dr - beta * del1) / alpha;
    const double delta = er / alpha;
    at(A.ia, r) = 1.0 / alpha;
    at(A.bb, r) = beta / alpha;
    at(A.ee, r) = ar / alpha;
    at(A.ga, r) = gamma;
    at(A.de, r) = delta;
    gam2 = gam1;
    del2 = del1;
    gam1 = gamma;
    del1 = delta;
  }
  if (failed) {  // leave a finite, harmless reduction behind: identity E, zero couplings
    for (int64_t r = 0; r < m; ++r) {
      at(A.ia, r) = 1.0;
      at(A.bb, r) = at(A.ee, r) = at(A.ga, r) = at(A.de, r) = 0.0;
      at(A.z0, r) = at(A.z1, r) = at(A.w0, r) = at(A.w1, r) = 0.0;
    }
    A.sinv[4 * s + 0] = A.sinv[4 * s + 3] = 1.0;
    A.sinv[4 * s + 1] = A.sinv[4 * s + 2] = 0.0;
    return;
  }
  // ---- the coupling blocks (rows of A listed by the column they reach) ----
  double a0, b0, c0, d0, e0, a1, b1, c1, d1, e1, am2, bm2, cm2, dm2, em2, am1, bm1, cm1, dm1, em1;
  double an2, bn2, cn2, dn2, en2, an1, bn1, cn1, dn1, en1;
  cyc_band(A, s, 0, a, b, c, d, e, sigma, a0, b0, c0, d0, e0);
  cyc_band(A, s, 1, a, b, c, d, e, sigma, a1, b1, c1, d1, e1);
  cyc_band(A, s, m - 2, a, b, c, d, e, sigma, am2, bm2, cm2, dm2, em2);
  cyc_band(A, s, m - 1, a, b, c, d, e, sigma, am1, bm1, cm1, dm1, em1);
  cyc_band(A, s, n - 2, a, b, c, d, e, sigma, an2, bn2, cn2, dn2, en2);
  cyc_band(A, s, n - 1, a, b, c, d, e, sigma, an1, bn1, cn1, dn1, en1);
  // k (columns n-2, n-1 of rows 0..m-1): nonzero in rows 0, 1, m-2, m-1
  auto k0 = [&](int64_t r) { return (r == 0 ? a0 : 0.0) + (r == m - 2 ? em2 : 0.0) + (r == m - 1 ? dm1 : 0.0); };
  auto k1 = [&](int64_t r) { return (r == 0 ? b0 : 0.0) + (r == 1 ? a1 : 0.0) + (r == m - 1 ? em1 : 0.0); };
  // h^T (rows n-2, n-1 restricted to columns 0..m-1): nonzero in columns 0, 1, m-2, m-1
  auto h0 = [&](int64_t r) { return (r == 0 ? en2 : 0.0) + (r == m - 2 ? an2 : 0.0) + (r == m - 1 ? bn2 : 0.0); };
  auto h1 = [&](int64_t r) { return (r == 0 ? dn1 : 0.0) + (r == 1 ? en1 : 0.0) + (r == m - 1 ? an1 : 0.0); };
  // ---- W = L^{-1} k: forward substitution with the stored records ----
  {
    double p2 = 0.0, p1 = 0.0, q2 = 0.0, q1 = 0.0;
    for (int64_t r = 0; r < m; ++r) {
      const double ia = at(A.ia, r), bb = at(A.bb, r), ee = at(A.ee, r);
      const double w0 = fma(-bb, p1, fma(-ee, p2, ia * k0(r)));
      const double w1 = fma(-bb, q1, fma(-ee, q2, ia * k1(r)));
      at(A.w0, r) = w0;
      at(A.w1, r) = w1;
      p2 = p1;
      p1 = w0;
      q2 = q1;
      q1 = w1;
    }
  }
  // ---- Z = E^{-T} h: R^T u = h (unit lower), then L^T z = u ----
  {
    double p2 = 0.0, p1 = 0.0, q2 = 0.0, q1 = 0.0;  // u_{r-2}, u_{r-1} of both columns
    double gm1 = 0.0, dm1x = 0.0, dm2x = 0.0;          // gamma_{r-1}, delta_{r-1}, delta_{r-2}
    for (int64_t r = 0; r < m; ++r) {
      const double u0 = h0(r) - gm1 * p1 - dm2x * p2;
      const double u1 = h1(r) - gm1 * q1 - dm2x * q2;
      at(A.z0, r) = u0;
      at(A.z1, r) = u1;
      p2 = p1;
      p1 = u0;
      q2 = q1;
      q1 = u1;
      dm2x = dm1x;
      gm1 = at(A.ga, r);
      dm1x = at(A.de, r);
    }
    // L^T z = u: alpha_r z_r + beta_{r+1} z_{r+1} + epsilon_{r+2} z_{r+2} = u_r
    double z1a = 0.0, z2a = 0.0, z1b = 0.0, z2b = 0.0;  // z_{r+1}, z_{r+2} of both columns
    for (int64_t r = m - 1; r >= 0; --r) {
      const double ia = at(A.ia, r);
      const double bnext = (r + 1 < m) ? at(A.bb, r + 1) / at(A.ia, r + 1) : 0.0;  // beta_{r+1}
      const double enext = (r + 2 < m) ? at(A.ee, r + 2) / at(A.ia, r + 2) : 0.0;  // epsilon_{r+2}
      const double za = ia * (at(A.z0, r) - bnext * z1a - enext * z2a);
      const double zb = ia * (at(A.z1, r) - bnext * z1b - enext * z2b);
      at(A.z0, r) = za;
      at(A.z1, r) = zb;
      z2a = z1a;
      z1a = za;
      z2b = z1b;
      z1b = zb;
    }
  }
  // ---- S = D - h^T E^{-1} k = D - Z^T k, and its inverse ----
  double s00 = cn2, s01 = dn2, s10 = bn1, s11 = cn1;
  const int64_t rows[4] = {0, 1, m - 2, m - 1};
  for (int j = 0; j < 4; ++j) {
    const int64_t r = rows[j];
    if (j == 2 && m - 2 <= 1) continue;  // row already counted (m = 3: m - 2 = 1)
    if (j == 3 && m - 1 <= 1) continue;
    const double z0 = at(A.z0, r), z1 = at(A.z1, r), kk0 = k0(r), kk1 = k1(r);
    s00 -= z0 * kk0;
    s01 -= z0 * kk1;
    s10 -= z1 * kk0;
    s11 -= z1 * kk1;
  }
  const double det = s00 * s11 - s01 * s10;
  if (!(det != 0.0) || !isfinite(det)) {
    report_bad(A.info, s, n - 2);
    A.sinv[4 * s + 0] = A.sinv[4 * s + 3] = 1.0;
    A.sinv[4 * s + 1] = A.sinv[4 * s + 2] = 0.0;
    return;
  }
  A.sinv[4 * s + 0] = s11 / det;
  A.sinv[4 * s + 1] = -s01 / det;
  A.sinv[4 * s + 2] = -s10 / det;
  A.sinv[4 * s + 3] = s00 / det;
}

// Explicit part of a periodic time step at row i from the window C_{i-2..i+2}:
//   f_i = C_i + mu (D2 (C^3 - C))_i - nu (D4 C)_i
// (Crank-Nicolson, Eq. matrix_sys: mu = 0, nu = sigma_x; Cahn-Hilliard,
// Eq. temporal: nu = 0, mu = D dt / dx^2).
__device__ __forceinline__ double rhs_row(double cm2, double cm1, double c0, double cp1, double cp2, double mu,
                                          double nu) {
  double f = c0;
  if (nu != 0.0) f = fma(-nu, fma(6.0, c0, fma(-4.0, cm1 + cp1, cm2 + cp2)), f);
  if (mu != 0.0) {
    const double um1 = fma(cm1 * cm1, cm1, -cm1), u0 = fma(c0 * c0, c0, -c0), up1 = fma(cp1 * cp1, cp1, -cp1);
    f = fma(mu, fma(-2.0, u0, um1 + up1), f);
  }
  return f;
}

// One thread per system: forward sweep over E's rows with the dot products
// Z^T f-hat, the 2x2 solve for the last two unknowns (Eq. first_two), then the
// back sweep on g - W t (Eq. solve).  RHS: f is assembled from the field in
// `f` (the old C) with per-system mu, nu.  x may alias f.
template <bool SHARED, bool RHS>
__global__ void __launch_bounds__(128) k_solve_periodic(PerArgs A, const double* f, double* x,
                                                        const double* __restrict__ mu_s,
                                                        const double* __restrict__ nu_s) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= A.batch) return;
  const int64_t n = A.n, m = A.m;
  const int64_t S = SHARED ? 1 : A.batch;
  const int64_t sr = SHARED ? 0 : s;
  auto rec = [&](const double* p, int64_t r) { return __ldg(p + r * S + sr); };
  const double* fs = f + s * n;
  double* xs = x + s * n;
  double mu = 0.0, nu = 0.0;
  if (RHS) {
    mu = mu_s ? mu_s[SHARED ? 0 : s] : 0.0;
    nu = nu_s ? nu_s[SHARED ? 0 : s] : 0.0;
  }
  // window of the old field (RHS): w0..w4 = C_{i-2} .. C_{i+2}
  double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0, w4 = 0.0, c0s = 0.0, c1s = 0.0;
  if (RHS) {
    w0 = fs[n - 2];
    w1 = fs[n - 1];
    w2 = c0s = fs[0];
    w3 = c1s = fs[1];
    w4 = fs[2];
  }
  // ---- forward: L g = f-hat, with Z^T f-hat ----
  double g1 = 0.0, g2 = 0.0, acc0 = 0.0, acc1 = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    double fi;
    if (RHS) {
      fi = rhs_row(w0, w1, w2, w3, w4, mu, nu);
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = w4;
      const int64_t j = i + 3;  // <= n: row n wraps to row 0
      w4 = (j < n) ? fs[j] : c0s;
    } else {
      fi = fs[i];
    }
    const double g = fma(-rec(A.bb, i), g1, fma(-rec(A.ee, i), g2, rec(A.ia, i) * fi));
    A.gscr[i * A.batch + s] = g;
    acc0 = fma(rec(A.z0, i), fi, acc0);
    acc1 = fma(rec(A.z1, i), fi, acc1);
    g2 = g1;
    g1 = g;
  }
  // ---- the last two unknowns (Eq. first_two) ----
  double fa, fb;
  if (RHS) {
    fa = rhs_row(w0, w1, w2, w3, w4, mu, nu);  // row n - 2: window C_{n-4} .. C_{n-1}, C_0
    w0 = w1;
    w1 = w2;
    w2 = w3;
    w3 = w4;
    w4 = c1s;                                   // C_{n+1} = C_1
    fb = rhs_row(w0, w1, w2, w3, w4, mu, nu);  // row n - 1
  } else {
    fa = fs[n - 2];
    fb = fs[n - 1];
  }
  const double2 s01 = *reinterpret_cast<const double2*>(A.sinv + 4 * sr);
  const double2 s23 = *reinterpret_cast<const double2*>(A.sinv + 4 * sr + 2);
  const double t0 = fa - acc0, t1 = fb - acc1;
  const double xa = fma(s01.x, t0, s01.y * t1);
  const double xb = fma(s23.x, t0, s23.y * t1);
  // ---- back: R X = g - W t ----
  double x1 = 0.0, x2 = 0.0;
  for (int64_t i = m - 1; i >= 0; --i) {
    const double gg = fma(-rec(A.w0, i), xa, fma(-rec(A.w1, i), xb, A.gscr[i * A.batch + s]));
    const double xv = fma(-rec(A.ga, i), x1, fma(-rec(A.de, i), x2, gg));
    xs[i] = xv;
    x2 = x1;
    x1 = xv;
  }
  xs[n - 2] = xa;
  xs[n - 1] = xb;
}

}  // namespace

cudaError_t launch_factor_periodic(const PerArgs& A, const double* a, const double* b, const double* c,
                                   const double* d, const double* e, const double* sigma, cudaStream_t st) {
  const int64_t S = A.shared ? 1 : A.batch;
  const int block = 128;
  k_factor_periodic<<<(unsigned)((S + block - 1) / block), block, 0, st>>>(A, a, b, c, d, e, sigma);
  return cudaGetLastError();
}

cudaError_t launch_solve_periodic(const PerArgs& A, const double* f, double* x, const double* mu, const double* nu,
                                  bool rhs, cudaStream_t st) {
  const int block = 128;
  const unsigned grid = (unsigned)((A.batch + block - 1) / block);
  if (A.shared) {
    if (rhs)
      k_solve_periodic<true, true><<<grid, block, 0, st>>>(A, f, x, mu, nu);
    else
      k_solve_periodic<true, false><<<grid, block, 0, st>>>(A, f, x, mu, nu);
  } else {
    if (rhs)
      k_solve_periodic<false, true><<<grid, block, 0, st>>>(A, f, x, mu, nu);
    else
      k_solve_periodic<false, false><<<grid, block, 0, st>>>(A, f, x, mu, nu);
  }
  return cudaGetLastError();
}

}  // namespace pent
