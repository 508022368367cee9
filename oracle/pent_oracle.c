/*
 * CPU oracle for the batched pentadiagonal factor-once / solve-many method of
 * Gloster, O Naraigh and Pang, "cuPentBatch -- A batched pentadiagonal solver
 * for NVIDIA GPUs" (arXiv 1807.07382).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  It is the plain, serial, FP64 restatement
 * of what the GPU library computes, and it exists only so that the tests, the
 * library's smoke check and the benchmark's CPU-baseline leg can check and time
 * the CUDA path against it.  The CUDA library never links, loads or calls it,
 * and it shares no code, header or table with the CUDA library.
 *
 * Indexing: C arrays are 0-based; array index i holds the paper's row i+1.
 * A row's band is (a_i, b_i, c_i, d_i, e_i), the coefficients of
 * x_{i-2}, x_{i-1}, x_i, x_{i+1}, x_{i+2} (Sec. 2.4, the matrix A before the
 * factorisation steps).  Entries that would fall outside the matrix are never
 * read; quantities with an index outside 0..n-1 are taken as zero.
 *
 * Batched entry points loop over systems with an OpenMP parallel for, which is
 * how the paper's OpenMP comparison code parallelises its serial solver
 * (Sec. 3.3); each system is still solved serially by one thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int po_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Band of the implicit hyperdiffusion matrix.                               */
/* ------------------------------------------------------------------------ */

/*
 * Band of D4, the centred fourth difference C_{i-2} - 4C_{i-1} + 6C_i -
 * 4C_{i+1} + C_{i+2} (Sec. 2.2, the discretised hyperdiffusion equation).
 * The paper's grid is periodic; the workloads here use a no-flux wall
 * instead, read as a cell-centred grid with even reflection (C_{-1} = C_0,
 * C_{-2} = C_1 and the mirror image at the right end).  Under that reflection
 * D4 is exactly the square of the no-flux second difference
 * D2N = tridiag(1, -2, 1) whose first and last diagonal entries are -1, and
 * this function builds D4 by multiplying out D2N * D2N.  All entries are
 * small integers.  Valid for any n >= 1.
 */
void po_band_d4(int64_t n, double* a, double* b, double* c, double* d, double* e) {
  for (int64_t i = 0; i < n; ++i) {
    /* D2N entries around row k: L_(k) = D2N[k][k-1], M_(k) = D2N[k][k], U_(k) = D2N[k][k+1] */
#define L_(k) (((k) >= 1 && (k) < n) ? 1.0 : 0.0)
#define U_(k) (((k) >= 0 && (k) + 1 < n) ? 1.0 : 0.0)
#define M_(k) (((k) >= 0 && (k) < n) ? (-2.0 + ((k) == 0 ? 1.0 : 0.0) + ((k) == n - 1 ? 1.0 : 0.0)) : 0.0)
    a[i] = L_(i) * L_(i - 1);                                  /* (D2N^2)[i][i-2] */
    b[i] = L_(i) * M_(i - 1) + M_(i) * L_(i);                  /* (D2N^2)[i][i-1] */
    c[i] = L_(i) * U_(i - 1) + M_(i) * M_(i) + U_(i) * L_(i + 1); /* (D2N^2)[i][i] */
    d[i] = M_(i) * U_(i) + U_(i) * M_(i + 1);                  /* (D2N^2)[i][i+1] */
    e[i] = U_(i) * U_(i + 1);                                  /* (D2N^2)[i][i+2] */
#undef L_
#undef U_
#undef M_
  }
}

/*
 * A = I + sigma * D4: the implicit-Euler hyperdiffusion matrix.  With the
 * periodic grid and Crank-Nicolson weighting of Sec. 2.2-2.3 the same band
 * reads a = e = sigma_x, b = d = -4 sigma_x, c = 1 + 6 sigma_x in the
 * interior; the workloads here step implicitly, so sigma multiplies the
 * whole of D4.
 */
void po_band_hyperdiff(int64_t n, double sigma, double* a, double* b, double* c, double* d, double* e) {
  po_band_d4(n, a, b, c, d, e);
  for (int64_t i = 0; i < n; ++i) {
    a[i] = sigma * a[i];
    b[i] = sigma * b[i];
    c[i] = 1.0 + sigma * c[i];
    d[i] = sigma * d[i];
    e[i] = sigma * e[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Factorisation A = L R and substitution (Sec. 2.4).                        */
/* ------------------------------------------------------------------------ */

/*
 * Factor A = L R without pivoting (Sec. 2.4, factorisation steps 1-14).
 * L is lower triangular with diagonal alpha, first subdiagonal beta and second
 * subdiagonal epsilon; R is unit upper triangular with superdiagonals gamma
 * and delta.  The loop is the paper's generic step for rows 3..N-2; with the
 * out-of-range quantities equal to zero it also reproduces the paper's special
 * first two and last two rows.  Returns -1, or the first row whose pivot
 * alpha is zero or not finite (the paper does not pivot, so such a system has
 * no factorisation of this form).
 */
int64_t po_factor(int64_t n, const double* a, const double* b, const double* c, const double* d, const double* e,
                  double* alpha, double* beta, double* gamma, double* delta, double* eps) {
  for (int64_t i = 0; i < n; ++i) {
    const double a_i = (i >= 2) ? a[i] : 0.0;
    const double b_i = (i >= 1) ? b[i] : 0.0;
    const double d_i = (i + 1 < n) ? d[i] : 0.0;
    const double e_i = (i + 2 < n) ? e[i] : 0.0;
    const double gamma_im2 = (i >= 2) ? gamma[i - 2] : 0.0;
    const double delta_im2 = (i >= 2) ? delta[i - 2] : 0.0;
    const double gamma_im1 = (i >= 1) ? gamma[i - 1] : 0.0;
    const double delta_im1 = (i >= 1) ? delta[i - 1] : 0.0;

    beta[i] = b_i - a_i * gamma_im2;                          /* beta_i  = b_i - a_i gamma_{i-2} */
    alpha[i] = c[i] - a_i * delta_im2 - beta[i] * gamma_im1;  /* alpha_i = c_i - a_i delta_{i-2} - beta_i gamma_{i-1} */
    if (!(alpha[i] != 0.0) || !isfinite(alpha[i])) return i;
    gamma[i] = (d_i - beta[i] * delta_im1) / alpha[i];        /* gamma_i = (d_i - beta_i delta_{i-1}) / alpha_i */
    delta[i] = e_i / alpha[i];                                /* delta_i = e_i / alpha_i */
    eps[i] = a_i;                                             /* epsilon_i = a_i */
  }
  return -1;
}

/*
 * Solve A x = f from the factors (Sec. 2.4): forward substitution L g = f,
 *   g_i = (f_i - epsilon_i g_{i-2} - beta_i g_{i-1}) / alpha_i,
 * then back substitution R x = g,
 *   x_i = g_i - gamma_i x_{i+1} - delta_i x_{i+2}.
 * `g` is caller-provided scratch of n doubles; x may alias f.
 */
void po_solve(int64_t n, const double* alpha, const double* beta, const double* gamma, const double* delta,
              const double* eps, const double* f, double* x, double* g) {
  for (int64_t i = 0; i < n; ++i) {
    double s = f[i];
    if (i >= 2) s -= eps[i] * g[i - 2];
    if (i >= 1) s -= beta[i] * g[i - 1];
    g[i] = s / alpha[i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = g[i];
    if (i + 1 < n) s -= gamma[i] * x[i + 1];
    if (i + 2 < n) s -= delta[i] * x[i + 2];
    x[i] = s;
  }
}

/*
 * Band of the transpose: row i of A^T holds column i of A, so
 * a'_i = e_{i-2}, b'_i = d_{i-1}, c'_i = c_i, d'_i = b_{i+1}, e'_i = a_{i+2}.
 */
void po_transpose_band(int64_t n, const double* a, const double* b, const double* c, const double* d, const double* e,
                       double* at, double* bt, double* ct, double* dt, double* et) {
  for (int64_t i = 0; i < n; ++i) {
    at[i] = (i >= 2) ? e[i - 2] : 0.0;
    bt[i] = (i >= 1) ? d[i - 1] : 0.0;
    ct[i] = c[i];
    dt[i] = (i + 1 < n) ? b[i + 1] : 0.0;
    et[i] = (i + 2 < n) ? a[i + 2] : 0.0;
  }
}

/* y = A x for one system (the definition of the band). */
void po_matvec(int64_t n, const double* a, const double* b, const double* c, const double* d, const double* e,
               const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = c[i] * x[i];
    if (i >= 2) s += a[i] * x[i - 2];
    if (i >= 1) s += b[i] * x[i - 1];
    if (i + 1 < n) s += d[i] * x[i + 1];
    if (i + 2 < n) s += e[i] * x[i + 2];
    y[i] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Batched drivers.  off[s] .. off[s+1]-1 are the rows of system s.          */
/* ------------------------------------------------------------------------ */

/* Factor every system; returns -1 or the lowest failing system index, whose
 * failing row goes to *bad_row. */
int64_t po_factor_batch(int64_t batch, const int64_t* off, const double* a, const double* b, const double* c,
                        const double* d, const double* e, double* alpha, double* beta, double* gamma, double* delta,
                        double* eps, int nthreads, int64_t* bad_row) {
  int64_t bad_sys = -1, bad_r = -1;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t o = off[s], n = off[s + 1] - off[s];
    int64_t r = po_factor(n, a + o, b + o, c + o, d + o, e + o, alpha + o, beta + o, gamma + o, delta + o, eps + o);
    if (r >= 0) {
#pragma omp critical
      {
        if (bad_sys < 0 || s < bad_sys) { bad_sys = s; bad_r = r; }
      }
    }
  }
  if (bad_row) *bad_row = bad_r;
  return bad_sys;
}

/* x_s = A_s^{-1} f_s for every system (x may alias f). */
void po_solve_batch(int64_t batch, const int64_t* off, const double* alpha, const double* beta, const double* gamma,
                    const double* delta, const double* eps, const double* f, double* x, int nthreads) {
  set_threads(nthreads);
#pragma omp parallel
  {
    int64_t cap = 0;
    double* g = NULL;
#pragma omp for schedule(dynamic, 16)
    for (int64_t s = 0; s < batch; ++s) {
      const int64_t o = off[s], n = off[s + 1] - off[s];
      if (n > cap) { free(g); cap = n; g = (double*)malloc((size_t)cap * sizeof(double)); }
      po_solve(n, alpha + o, beta + o, gamma + o, delta + o, eps + o, f + o, x + o, g);
    }
    free(g);
  }
}

/*
 * Solve A^T y = f for one system from the band of A (the adjoint solve).  The
 * oracle takes the plain definition: it forms the transposed band and applies
 * the factorisation and substitutions of Sec. 2.4 to it.  `work` holds 11 n
 * doubles.  Returns -1 or the failing row of the transposed factorisation.
 */
int64_t po_adjoint_solve(int64_t n, const double* a, const double* b, const double* c, const double* d,
                         const double* e, const double* f, double* y, double* work) {
  double *at = work, *bt = work + n, *ct = work + 2 * n, *dt = work + 3 * n, *et = work + 4 * n;
  double *al = work + 5 * n, *be = work + 6 * n, *ga = work + 7 * n, *de = work + 8 * n, *ep = work + 9 * n;
  double* g = work + 10 * n;
  po_transpose_band(n, a, b, c, d, e, at, bt, ct, dt, et);
  int64_t r = po_factor(n, at, bt, ct, dt, et, al, be, ga, de, ep);
  if (r < 0) po_solve(n, al, be, ga, de, ep, f, y, g);
  return r;
}

/* Adjoint solve for every system; returns -1 or the lowest failing system. */
int64_t po_adjoint_solve_batch(int64_t batch, const int64_t* off, const double* a, const double* b, const double* c,
                               const double* d, const double* e, const double* f, double* y, int nthreads) {
  int64_t bad_sys = -1;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t o = off[s], n = off[s + 1] - off[s];
    double* w = (double*)malloc((size_t)11 * (size_t)(n > 0 ? n : 1) * sizeof(double));
    if (po_adjoint_solve(n, a + o, b + o, c + o, d + o, e + o, f + o, y + o, w) >= 0) {
#pragma omp critical
      {
        if (bad_sys < 0 || s < bad_sys) bad_sys = s;
      }
    }
    free(w);
  }
  return bad_sys;
}

/*
 * `steps` implicit-Euler hyperdiffusion steps (I + sigma_s D4) C^{k+1} = C^k on
 * every system, in place on `field` (system-major).  sigma has `batch` entries,
 * or one entry shared by all systems when shared != 0.  Each system's matrix
 * is built and factored once and reused for every step (the paper's
 * factor-once, solve-many use, Sec. 2.6).
 */
int64_t po_hyperdiff_steps(int64_t batch, const int64_t* off, const double* sigma, int shared, int64_t steps,
                           double* field, int nthreads) {
  int64_t bad_sys = -1;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t o = off[s], n = off[s + 1] - off[s];
    const double sg = shared ? sigma[0] : sigma[s];
    double* w = (double*)malloc((size_t)11 * (size_t)(n > 0 ? n : 1) * sizeof(double));
    double *a = w, *b = w + n, *c = w + 2 * n, *d = w + 3 * n, *e = w + 4 * n;
    double *al = w + 5 * n, *be = w + 6 * n, *ga = w + 7 * n, *de = w + 8 * n, *ep = w + 9 * n, *g = w + 10 * n;
    po_band_hyperdiff(n, sg, a, b, c, d, e);
    if (po_factor(n, a, b, c, d, e, al, be, ga, de, ep) >= 0) {
#pragma omp critical
      {
        if (bad_sys < 0 || s < bad_sys) bad_sys = s;
      }
    } else {
      for (int64_t k = 0; k < steps; ++k) po_solve(n, al, be, ga, de, ep, field + o, field + o, g);
    }
    free(w);
  }
  return bad_sys;
}

/* ------------------------------------------------------------------------ */
/* Two-dimensional Cahn-Hilliard step by alternating directions (Sec. 4).    */
/* ------------------------------------------------------------------------ */

/*
 * out = L v for the five-point Laplacian in grid units, L = D2N_x + D2N_y,
 * with the same cell-centred no-flux reflection as the 1D band (the ghost
 * value beyond a wall equals the cell next to the wall).  v and out are
 * ny x nx, row-major (x fastest).
 */
void po_laplacian_noflux(int64_t nx, int64_t ny, const double* v, double* out) {
  for (int64_t y = 0; y < ny; ++y) {
    for (int64_t x = 0; x < nx; ++x) {
      const double c0 = v[y * nx + x];
      const double w = (x > 0) ? v[y * nx + x - 1] : c0;
      const double ea = (x + 1 < nx) ? v[y * nx + x + 1] : c0;
      const double s = (y > 0) ? v[(y - 1) * nx + x] : c0;
      const double nn = (y + 1 < ny) ? v[(y + 1) * nx + x] : c0;
      out[y * nx + x] = (w - 2.0 * c0 + ea) + (s - 2.0 * c0 + nn);
    }
  }
}

/*
 * Right-hand side of the delta-form step:
 *   rhs = mu * L(C^3 - C) - sigma * L(L C),
 * mu = dt/dx^2, sigma = gamma dt/dx^4.  This is dt times the explicit part of
 * the semi-implicit Cahn-Hilliard scheme (Sec. 2.1, the time discretisation
 * with D = 1), with the implicit fourth-order operator written at the old
 * time level, as the delta form requires.
 */
void po_ch_rhs(int64_t nx, int64_t ny, const double* C, double mu, double sigma, double* rhs) {
  const size_t m = (size_t)nx * (size_t)ny;
  double* u = (double*)calloc(m > 0 ? m : 1, sizeof(double));
  double* lu = (double*)malloc(m * sizeof(double));
  double* lc = (double*)malloc(m * sizeof(double));
  double* llc = (double*)malloc(m * sizeof(double));
  for (size_t k = 0; k < m; ++k) u[k] = C[k] * C[k] * C[k] - C[k];
  po_laplacian_noflux(nx, ny, u, lu);
  po_laplacian_noflux(nx, ny, C, lc);
  po_laplacian_noflux(nx, ny, lc, llc);
  for (size_t k = 0; k < m; ++k) rhs[k] = mu * lu[k] - sigma * llc[k];
  free(u); free(lu); free(lc); free(llc);
}

/*
 * Solve (I + sigma D4_x)(I + sigma D4_y) dC = rhs in place on rhs (ny x nx,
 * row-major): the x sweep solves one system of n = nx along every grid row,
 * then the y sweep one system of n = ny along every grid column.  Each sweep's
 * matrix is built and factored once and shared by all its systems.  Returns
 * -1 on success or 0/1 if the x/y matrix cannot be factored.
 */
int64_t po_adi_solve(int64_t nx, int64_t ny, double* rhs, double sigma, int nthreads) {
  int64_t status = -1;
  set_threads(nthreads);
  for (int dir = 0; dir < 2 && status < 0; ++dir) {
    const int64_t n = dir == 0 ? nx : ny;      /* system length */
    const int64_t count = dir == 0 ? ny : nx;  /* number of systems */
    double* w = (double*)malloc((size_t)10 * (size_t)n * sizeof(double));
    double *a = w, *b = w + n, *c = w + 2 * n, *d = w + 3 * n, *e = w + 4 * n;
    double *al = w + 5 * n, *be = w + 6 * n, *ga = w + 7 * n, *de = w + 8 * n, *ep = w + 9 * n;
    po_band_hyperdiff(n, sigma, a, b, c, d, e);
    if (po_factor(n, a, b, c, d, e, al, be, ga, de, ep) >= 0) {
      status = dir;
    } else {
#pragma omp parallel
      {
        double* line = (double*)malloc((size_t)n * sizeof(double));
        double* g = (double*)malloc((size_t)n * sizeof(double));
#pragma omp for
        for (int64_t s = 0; s < count; ++s) {
          for (int64_t k = 0; k < n; ++k) line[k] = dir == 0 ? rhs[s * nx + k] : rhs[k * nx + s];
          po_solve(n, al, be, ga, de, ep, line, line, g);
          for (int64_t k = 0; k < n; ++k) {
            if (dir == 0) rhs[s * nx + k] = line[k]; else rhs[k * nx + s] = line[k];
          }
        }
        free(line); free(g);
      }
    }
    free(w);
  }
  return status;
}

/*
 * One alternating-direction step of the 2D Cahn-Hilliard equation in the
 * Douglas delta form, in place on C (ny x nx, no-flux walls):
 *   (I + sigma D4_x)(I + sigma D4_y) dC = mu L(C^3 - C) - sigma L(L C),
 *   dC <- dC - mean(dC),   C <- C + dC.
 * The paper only states that the 2D implicit matrix reduces to 1D
 * pentadiagonal problems by ADI (Sec. 4, citing Douglas 1955); the scheme
 * above is this library's reading of that remark.  In exact arithmetic dC has
 * zero mean (L has zero column sums and each implicit factor unit column
 * sums), so subtracting the mean removes only the rounding of the large
 * O(sigma) right-hand side in the constant mode, which would otherwise show
 * up as a drift of the total mass.  Returns -1 on success.
 */
int64_t po_adi_step_ms(int64_t nx, int64_t ny, double* C, double mu, double sigma, int nthreads) {
  const size_t m = (size_t)nx * (size_t)ny;
  double* rhs = (double*)malloc((m > 0 ? m : 1) * sizeof(double));
  po_ch_rhs(nx, ny, C, mu, sigma, rhs);
  int64_t status = po_adi_solve(nx, ny, rhs, sigma, nthreads);
  if (status < 0 && m > 0) {
    double sum = 0.0;
    for (size_t k = 0; k < m; ++k) sum += rhs[k];
    const double mean = sum / (double)m;
    for (size_t k = 0; k < m; ++k) C[k] += rhs[k] - mean;
  }
  free(rhs);
  return status;
}

/* The same step from the physical parameters: mu = dt/dx^2, sigma = gamma dt/dx^4. */
int64_t po_adi_step(int64_t nx, int64_t ny, double* C, double gamma, double dt, double dx, int nthreads) {
  const double mu = dt / (dx * dx);
  const double sigma = gamma * dt / (dx * dx * dx * dx);
  return po_adi_step_ms(nx, ny, C, mu, sigma, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Loss over T implicit steps and its gradient by the adjoint.               */
/* ------------------------------------------------------------------------ */

/*
 * Forward: x^0 = C0_s, (I + sigma_s D4) x^k = x^{k-1}, k = 1..T.
 * Loss: sum_s ||x_s^T - target_s||^2.
 * Gradient by the discrete adjoint: lambda^T = 2 (x^T - target); for k = T..1,
 *   mu^k = A^{-T} lambda^k,  dL/dsigma_s -= (mu^k)^T D4 x^k,  lambda^{k-1} = mu^k;
 * dL/dC0 = lambda^0.  (From A x^k = x^{k-1} and dA/dsigma = D4.)
 * The whole trajectory is kept (no checkpointing is needed on the CPU).
 * Returns the loss; grad_c0 / grad_sigma may be NULL.
 */
double po_hyperdiff_loss_grad(int64_t batch, int64_t n, const double* sigma, int64_t T, const double* c0,
                              const double* target, double* grad_c0, double* grad_sigma, int nthreads) {
  double loss = 0.0;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : loss)
  for (int64_t s = 0; s < batch; ++s) {
    const double sg = sigma[s];
    double* w = (double*)malloc((size_t)(35 + (T + 1)) * (size_t)n * sizeof(double));
    double *a = w, *b = w + n, *c = w + 2 * n, *d = w + 3 * n, *e = w + 4 * n;
    double *al = w + 5 * n, *be = w + 6 * n, *ga = w + 7 * n, *de = w + 8 * n, *ep = w + 9 * n, *g = w + 10 * n;
    double *lam = w + 11 * n, *mu = w + 12 * n, *d4x = w + 13 * n;
    double *qa = w + 14 * n, *qb = w + 15 * n, *qc = w + 16 * n, *qd = w + 17 * n, *qe = w + 18 * n;
    double* adj_work = w + 19 * n; /* 11 n */
    double* traj = w + 35 * n;     /* (T+1) x n */
    po_band_hyperdiff(n, sg, a, b, c, d, e);
    po_band_d4(n, qa, qb, qc, qd, qe);
    po_factor(n, a, b, c, d, e, al, be, ga, de, ep);
    memcpy(traj, c0 + s * n, (size_t)n * sizeof(double));
    for (int64_t k = 1; k <= T; ++k) po_solve(n, al, be, ga, de, ep, traj + (k - 1) * n, traj + k * n, g);
    double ls = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double r = traj[T * n + i] - target[s * n + i];
      ls += r * r;
      lam[i] = 2.0 * r;
    }
    loss += ls;
    double gs = 0.0;
    for (int64_t k = T; k >= 1; --k) {
      po_adjoint_solve(n, a, b, c, d, e, lam, mu, adj_work);
      po_matvec(n, qa, qb, qc, qd, qe, traj + k * n, d4x);
      for (int64_t i = 0; i < n; ++i) gs -= mu[i] * d4x[i];
      memcpy(lam, mu, (size_t)n * sizeof(double));
    }
    if (grad_c0) memcpy(grad_c0 + s * n, lam, (size_t)n * sizeof(double));
    if (grad_sigma) grad_sigma[s] = gs;
    free(w);
  }
  return loss;
}

/*
 * Vector-Jacobian product of the T-step map C0 -> x^T (same recurrences as
 * po_hyperdiff_loss_grad, with lambda^T supplied instead of formed from a
 * loss): returns dC0 = lambda^0 and dsigma_s = -sum_k mu^k . D4 x^k.
 */
void po_hyperdiff_vjp(int64_t batch, int64_t n, const double* sigma, int64_t T, const double* c0,
                      const double* lambda_T, double* grad_c0, double* grad_sigma, int nthreads) {
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t s = 0; s < batch; ++s) {
    const double sg = sigma[s];
    double* w = (double*)malloc((size_t)(35 + (T + 1)) * (size_t)n * sizeof(double));
    double *a = w, *b = w + n, *c = w + 2 * n, *d = w + 3 * n, *e = w + 4 * n;
    double *al = w + 5 * n, *be = w + 6 * n, *ga = w + 7 * n, *de = w + 8 * n, *ep = w + 9 * n, *g = w + 10 * n;
    double *lam = w + 11 * n, *mu = w + 12 * n, *d4x = w + 13 * n;
    double *qa = w + 14 * n, *qb = w + 15 * n, *qc = w + 16 * n, *qd = w + 17 * n, *qe = w + 18 * n;
    double* adj_work = w + 19 * n;
    double* traj = w + 35 * n;
    po_band_hyperdiff(n, sg, a, b, c, d, e);
    po_band_d4(n, qa, qb, qc, qd, qe);
    po_factor(n, a, b, c, d, e, al, be, ga, de, ep);
    memcpy(traj, c0 + s * n, (size_t)n * sizeof(double));
    for (int64_t k = 1; k <= T; ++k) po_solve(n, al, be, ga, de, ep, traj + (k - 1) * n, traj + k * n, g);
    memcpy(lam, lambda_T + s * n, (size_t)n * sizeof(double));
    double gs = 0.0;
    for (int64_t k = T; k >= 1; --k) {
      po_adjoint_solve(n, a, b, c, d, e, lam, mu, adj_work);
      po_matvec(n, qa, qb, qc, qd, qe, traj + k * n, d4x);
      for (int64_t i = 0; i < n; ++i) gs -= mu[i] * d4x[i];
      memcpy(lam, mu, (size_t)n * sizeof(double));
    }
    memcpy(grad_c0 + s * n, lam, (size_t)n * sizeof(double));
    grad_sigma[s] = gs;
    free(w);
  }
}

/* ------------------------------------------------------------------------ */
/* Periodic (cyclic) pentadiagonal systems: Navon's reduction (Sec. 2.3).    */
/* ------------------------------------------------------------------------ */

/*
 * Cyclic band: row i reads a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1}
 * + e_i x_{i+2} with every column index taken modulo n (Eq. matrix_sys1: the
 * corner entries a, b of the first rows and d, e of the last rows close the
 * period).  n >= 5, so the five columns of a row are distinct.
 */
void po_periodic_matvec(int64_t n, const double* a, const double* b, const double* c, const double* d,
                        const double* e, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    const int64_t im2 = (i + n - 2) % n, im1 = (i + n - 1) % n, ip1 = (i + 1) % n, ip2 = (i + 2) % n;
    y[i] = a[i] * x[im2] + b[i] * x[im1] + c[i] * x[i] + d[i] * x[ip1] + e[i] * x[ip2];
  }
}

/* The periodic hyperdiffusion matrix of Eq. (matrix_sys): a = e = sigma_x,
 * b = d = -4 sigma_x, c = 1 + 6 sigma_x on every row. */
void po_band_periodic_hyperdiff(int64_t n, double sigma, double* a, double* b, double* c, double* d, double* e) {
  for (int64_t i = 0; i < n; ++i) {
    a[i] = sigma;
    b[i] = -4.0 * sigma;
    c[i] = 1.0 + 6.0 * sigma;
    d[i] = -4.0 * sigma;
    e[i] = sigma;
  }
}

/*
 * Right-hand side of the Crank-Nicolson step, Eq. (matrix_sys):
 *   f_i = -sigma C_{i-2} + 4 sigma C_{i-1} + (1 - 6 sigma) C_i + 4 sigma C_{i+1} - sigma C_{i+2},
 * indices modulo n.
 */
void po_periodic_cn_rhs(int64_t n, double sigma, const double* C, double* f) {
  for (int64_t i = 0; i < n; ++i) {
    const int64_t im2 = (i + n - 2) % n, im1 = (i + n - 1) % n, ip1 = (i + 1) % n, ip2 = (i + 2) % n;
    f[i] = -sigma * C[im2] + 4.0 * sigma * C[im1] + (1.0 - 6.0 * sigma) * C[i] + 4.0 * sigma * C[ip1] -
           sigma * C[ip2];
  }
}

/*
 * Navon's reduction of a cyclic system, prepared once per matrix (Sec. 2.3:
 * the 2x2 inverse of Eq. (first_two) and the products with E^{-1} are formed
 * at the start and reused for every right-hand side).  With m = n - 2:
 *   E  = the leading m x m block of A (the last two rows and columns removed),
 *   k  = the m x 2 block of A in columns n-2, n-1 (paper: x_{N-1}, x_N),
 *   h^T = the 2 x m block of A in rows n-2, n-1,
 *   D  = the trailing 2 x 2 block [[c, d], [b, c]].
 * Stored: the factors of E (Sec. 2.4), Q = E^{-1} k (two columns), and
 * S^{-1} = (D - h^T E^{-1} k)^{-1}.
 */
typedef struct {
  int64_t n, m;
  double *al, *be, *ga, *de, *ep; /* factors of E */
  double *k0, *k1;                /* columns of k */
  double *h0, *h1;                /* columns of h: h^T's rows n-2, n-1 */
  double *q0, *q1;                /* E^{-1} k */
  double *g;                      /* solve scratch */
  double Sinv[4];
  double* mem;
} po_navon;

static void po_navon_free(po_navon* P) { free(P->mem); P->mem = NULL; }

/* Returns -1, or the failing row: a row of E, or n-2 when the 2x2 Schur complement is singular. */
static int64_t po_navon_prepare(po_navon* P, int64_t n, const double* a, const double* b, const double* c,
                                const double* d, const double* e) {
  const int64_t m = n - 2;
  P->n = n;
  P->m = m;
  P->mem = (double*)calloc((size_t)16 * (size_t)m, sizeof(double));
  double* w = P->mem;
  double *Ea = w, *Eb = w + m, *Ec = w + 2 * m, *Ed = w + 3 * m, *Ee = w + 4 * m;
  P->al = w + 5 * m; P->be = w + 6 * m; P->ga = w + 7 * m; P->de = w + 8 * m; P->ep = w + 9 * m;
  P->k0 = w + 10 * m; P->k1 = w + 11 * m; P->h0 = w + 12 * m; P->h1 = w + 13 * m;
  P->q0 = w + 14 * m; P->q1 = w + 15 * m;
  /* E: rows 0..m-1 of A restricted to columns 0..m-1 (po_factor ignores the out-of-range entries) */
  for (int64_t i = 0; i < m; ++i) { Ea[i] = a[i]; Eb[i] = b[i]; Ec[i] = c[i]; Ed[i] = d[i]; Ee[i] = e[i]; }
  /* k: the entries of rows 0..m-1 in columns n-2 and n-1 */
  P->k0[0] += a[0];          /* row 0, column (0 - 2) mod n = n-2 */
  P->k1[0] += b[0];          /* row 0, column n-1 */
  P->k1[1] += a[1];          /* row 1, column n-1 */
  P->k0[m - 2] += e[m - 2];  /* row m-2, column m = n-2 */
  P->k0[m - 1] += d[m - 1];  /* row m-1, column n-2 */
  P->k1[m - 1] += e[m - 1];  /* row m-1, column n-1 */
  /* h^T: the entries of rows n-2 and n-1 in columns 0..m-1 */
  P->h0[m - 2] += a[n - 2];  /* row n-2, column n-4 = m-2 */
  P->h0[m - 1] += b[n - 2];  /* row n-2, column m-1 */
  P->h0[0] += e[n - 2];      /* row n-2, column n mod n = 0 */
  P->h1[m - 1] += a[n - 1];  /* row n-1, column m-1 */
  P->h1[0] += d[n - 1];      /* row n-1, column 0 */
  P->h1[1] += e[n - 1];      /* row n-1, column 1 */
  const int64_t r = po_factor(m, Ea, Eb, Ec, Ed, Ee, P->al, P->be, P->ga, P->de, P->ep);
  if (r >= 0) return r;
  P->g = Ea; /* the band copy is no longer needed: reuse it as scratch */
  po_solve(m, P->al, P->be, P->ga, P->de, P->ep, P->k0, P->q0, P->g);
  po_solve(m, P->al, P->be, P->ga, P->de, P->ep, P->k1, P->q1, P->g);
  /* S = D - h^T E^{-1} k */
  double s00 = c[n - 2], s01 = d[n - 2], s10 = b[n - 1], s11 = c[n - 1];
  for (int64_t i = 0; i < m; ++i) {
    s00 -= P->h0[i] * P->q0[i];
    s01 -= P->h0[i] * P->q1[i];
    s10 -= P->h1[i] * P->q0[i];
    s11 -= P->h1[i] * P->q1[i];
  }
  const double det = s00 * s11 - s01 * s10;
  if (!(det != 0.0) || !isfinite(det)) return n - 2;
  P->Sinv[0] = s11 / det;
  P->Sinv[1] = -s01 / det;
  P->Sinv[2] = -s10 / det;
  P->Sinv[3] = s00 / det;
  return -1;
}

/* One right-hand side: Eq. (first_two) for x_{n-2}, x_{n-1}, then Eq. (solve) for the rest.
 * x may alias f; y is scratch of m doubles. */
static void po_navon_apply(const po_navon* P, const double* f, double* x, double* y) {
  const int64_t n = P->n, m = P->m;
  po_solve(m, P->al, P->be, P->ga, P->de, P->ep, f, y, P->g); /* E^{-1} f-hat */
  double t0 = f[n - 2], t1 = f[n - 1];
  for (int64_t i = 0; i < m; ++i) {
    t0 -= P->h0[i] * y[i];
    t1 -= P->h1[i] * y[i];
  }
  const double xa = P->Sinv[0] * t0 + P->Sinv[1] * t1;
  const double xb = P->Sinv[2] * t0 + P->Sinv[3] * t1;
  for (int64_t i = 0; i < m; ++i) y[i] = f[i] - P->k0[i] * xa - P->k1[i] * xb; /* f-hat - k x_tail */
  po_solve(m, P->al, P->be, P->ga, P->de, P->ep, y, x, P->g);
  x[n - 2] = xa;
  x[n - 1] = xb;
}

/* Solve one cyclic system A x = f (n >= 5).  Returns -1 or the failing row. */
int64_t po_periodic_solve(int64_t n, const double* a, const double* b, const double* c, const double* d,
                          const double* e, const double* f, double* x) {
  po_navon P;
  const int64_t r = po_navon_prepare(&P, n, a, b, c, d, e);
  if (r < 0) {
    double* y = (double*)malloc((size_t)(n - 2) * sizeof(double));
    po_navon_apply(&P, f, x, y);
    free(y);
  }
  po_navon_free(&P);
  return r;
}

/* Cyclic solve for every system of a batch of n-row systems (system-major). */
int64_t po_periodic_solve_batch(int64_t batch, int64_t n, const double* a, const double* b, const double* c,
                                const double* d, const double* e, const double* f, double* x, int nthreads) {
  int64_t bad_sys = -1;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t o = s * n;
    if (po_periodic_solve(n, a + o, b + o, c + o, d + o, e + o, f + o, x + o) >= 0) {
#pragma omp critical
      {
        if (bad_sys < 0 || s < bad_sys) bad_sys = s;
      }
    }
  }
  return bad_sys;
}

/*
 * `steps` periodic hyperdiffusion steps on every system, in place: each step
 * solves A C^{k+1} = f with A the matrix of Eq. (matrix_sys) and
 *   cn != 0: f = the Crank-Nicolson right-hand side of Eq. (matrix_sys),
 *   cn == 0: f = C^k (implicit Euler with the same matrix).
 * sigma: `batch` values (the paper's sigma_x = dt / (2 dx^4) for Crank-Nicolson),
 * or one shared value when shared != 0.  The reduction is prepared once per
 * system and reused for every step (Sec. 2.3).
 */
int64_t po_periodic_steps(int64_t batch, int64_t n, const double* sigma, int shared, int64_t steps, int cn,
                          double* field, int nthreads) {
  int64_t bad_sys = -1;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t s = 0; s < batch; ++s) {
    const double sg = shared ? sigma[0] : sigma[s];
    double* w = (double*)malloc((size_t)7 * (size_t)n * sizeof(double));
    double *a = w, *b = w + n, *c = w + 2 * n, *d = w + 3 * n, *e = w + 4 * n, *f = w + 5 * n, *y = w + 6 * n;
    po_band_periodic_hyperdiff(n, sg, a, b, c, d, e);
    po_navon P;
    if (po_navon_prepare(&P, n, a, b, c, d, e) >= 0) {
#pragma omp critical
      {
        if (bad_sys < 0 || s < bad_sys) bad_sys = s;
      }
    } else {
      double* C = field + s * n;
      for (int64_t k = 0; k < steps; ++k) {
        if (cn) po_periodic_cn_rhs(n, sg, C, f); else memcpy(f, C, (size_t)n * sizeof(double));
        po_navon_apply(&P, f, C, y);
      }
    }
    po_navon_free(&P);
    free(w);
  }
  return bad_sys;
}

/* ------------------------------------------------------------------------ */
/* Semi-implicit steps with an explicit part (Sec. 2.1 and 2.2).             */
/* ------------------------------------------------------------------------ */

/* Index j of an n-cell grid mapped into 0..n-1: by even reflection about the
 * cell-centred no-flux walls (periodic == 0), or modulo n (periodic != 0). */
static int64_t po_wrap(int64_t j, int64_t n, int periodic) {
  if (periodic) return ((j % n) + n) % n;
  while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
  return j;
}

/*
 * Explicit part of one step on an n-cell grid:
 *   f_i = C_i + mu (D2 (C^3 - C))_i - nu (D4 C)_i,
 * with the centred differences D2 = [1, -2, 1] and D4 = [1, -4, 6, -4, 1]
 * (Sec. 2.2) on the reflected (no-flux) or periodic grid.  mu = D dt / dx^2,
 * nu = 0 gives the right-hand side of the semi-implicit Cahn-Hilliard step of
 * Eq. (temporal); mu = 0, nu = sigma_x the Crank-Nicolson right-hand side of
 * Eq. (1d_hyper_scheme).  `u` is scratch of n doubles.
 */
void po_explicit_rhs(int64_t n, int periodic, double mu, double nu, const double* C, double* f, double* u) {
  for (int64_t i = 0; i < n; ++i) u[i] = C[i] * C[i] * C[i] - C[i];
  for (int64_t i = 0; i < n; ++i) {
    const double d2u = u[po_wrap(i - 1, n, periodic)] - 2.0 * u[i] + u[po_wrap(i + 1, n, periodic)];
    const double d4c = C[po_wrap(i - 2, n, periodic)] - 4.0 * C[po_wrap(i - 1, n, periodic)] + 6.0 * C[i] -
                       4.0 * C[po_wrap(i + 1, n, periodic)] + C[po_wrap(i + 2, n, periodic)];
    f[i] = C[i] + mu * d2u - nu * d4c;
  }
}

/*
 * `steps` steps (I + sigma_s D4) C^{k+1} = f(C^k) on every system, in place on
 * `field` (system-major), f the explicit part above with per-system mu_s, nu_s.
 * No-flux grid (periodic == 0): systems of sizes off[s+1] - off[s], the band
 * of po_band_hyperdiff, factored once (Sec. 2.4, 2.6).  Periodic grid: the
 * matrix of Eq. (matrix_sys) solved by Navon's reduction (Sec. 2.3).
 * sigma, mu, nu: `batch` values each, or one shared value when shared != 0;
 * mu or nu may be NULL for zero.
 */
int64_t po_explicit_steps(int64_t batch, const int64_t* off, int periodic, const double* sigma, const double* mu,
                          const double* nu, int shared, int64_t steps, double* field, int nthreads) {
  int64_t bad_sys = -1;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t s = 0; s < batch; ++s) {
    const int64_t o = off[s], n = off[s + 1] - off[s];
    const int64_t k = shared ? 0 : s;
    const double sg = sigma[k], m_ = mu ? mu[k] : 0.0, n_ = nu ? nu[k] : 0.0;
    double* w = (double*)malloc((size_t)13 * (size_t)(n > 0 ? n : 1) * sizeof(double));
    double *a = w, *b = w + n, *c = w + 2 * n, *d = w + 3 * n, *e = w + 4 * n;
    double *al = w + 5 * n, *be = w + 6 * n, *ga = w + 7 * n, *de = w + 8 * n, *ep = w + 9 * n;
    double *g = w + 10 * n, *f = w + 11 * n, *u = w + 12 * n;
    double* C = field + o;
    int ok;
    po_navon P;
    P.mem = NULL;
    if (periodic) {
      po_band_periodic_hyperdiff(n, sg, a, b, c, d, e);
      ok = po_navon_prepare(&P, n, a, b, c, d, e) < 0;
    } else {
      po_band_hyperdiff(n, sg, a, b, c, d, e);
      ok = po_factor(n, a, b, c, d, e, al, be, ga, de, ep) < 0;
    }
    if (!ok) {
#pragma omp critical
      {
        if (bad_sys < 0 || s < bad_sys) bad_sys = s;
      }
    } else {
      for (int64_t t = 0; t < steps; ++t) {
        po_explicit_rhs(n, periodic, m_, n_, C, f, u);
        if (periodic)
          po_navon_apply(&P, f, C, u);
        else
          po_solve(n, al, be, ga, de, ep, f, C, g);
      }
    }
    if (P.mem) po_navon_free(&P);
    free(w);
  }
  return bad_sys;
}
