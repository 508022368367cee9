// FP64 factorisation, substitution and adjoint kernels (one thread per system).
//
// Layout.  Systems are visited in "sorted position" order q = 0..ngroups*32-1
// (perm[q] is the system, longest first, so a warp's 32 systems have similar
// lengths).  Warp k owns the 32 systems q = 32k..32k+31 and walks the rows of
// all of them in lock step.  Record rows R = goff[k] + r (goff even, group
// lengths padded to even) are stored in pairs: for factor plane p the pair
// PR = R / 2 holds, for each lane, rows 2 PR and 2 PR + 1 side by side, so a
// warp fetches two rows of one plane for its 32 systems with one coalesced
// 512-byte access of 16 bytes per lane.  This is the interleaved
// one-thread-per-system layout of the paper (Sec. 2.6), applied per group of
// 32 systems (which keeps uneven lengths cheap to pad) and with row pairs (which
// halves the number of memory instructions per row).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace pent {
namespace {

// Weights of the centred fourth difference [1, -4, 6, -4, 1] (Sec. 2.2) on row
// i of an n-row cell-centred grid with no-flux walls: an index that falls
// outside 0..n-1 is reflected about the wall (-1 -> 0, -2 -> 1, n -> n-1,
// n+1 -> n-2, repeatedly for very short grids) and its weight is added to the
// reflected column.  w[k] is the coefficient of x_{i+k-2}.
__device__ __forceinline__ void d4_weights(int64_t i, int64_t n, double w[5]) {
  const double st[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = 0.0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    int64_t j = i + k - 2;
    while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
    const int64_t at = j - i + 2;  // within 0..4 for every row 0 <= i < n
    if (at >= 0 && at < 5) w[at] += st[k];
  }
}

__device__ __forceinline__ void report_bad_pivot(unsigned long long* info, int64_t s, int64_t r) {
  const unsigned long long key = ((unsigned long long)s << 32) | (unsigned long long)(uint32_t)r;
  atomicMin(info, key);
}

// Factor one system per thread (Sec. 2.4, factorisation steps 1-14, written as
// the generic row step with out-of-range quantities zero) and write its FP64
// records.  Rows after a failed pivot and padding rows get identity records
// (1/alpha = 1, all couplings 0), so later solves stay finite.  With F.sig the
// hyperdiffusion records are written instead (1/alpha and beta; epsilon is
// sigma), and those rows get 1/alpha = 0, which zeroes their g.
__global__ void k_factor64(DevPlan P, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ c, const double* __restrict__ d, const double* __restrict__ e,
                           const double* __restrict__ sigma, F64Factors F) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nslots = P.shared ? 1 : P.ngroups * kWarp;
  if (q >= nslots) return;
  const int64_t s = P.shared ? 0 : P.perm[q];
  const int64_t k = q / kWarp;
  const int lane = (int)(q % kWarp);
  const int64_t Lg = P.shared ? P.n_shared : P.glen[k];
  const int64_t R0 = P.shared ? 0 : P.goff[k];
  const bool hyp = !P.shared && F.sig != nullptr;
  const int np = hyp ? 2 : 3;
  auto fwd_at = [&](int64_t r, int p) -> double& {
    return P.shared ? F.fwd[r * 3 + p] : F.fwd[(((R0 + r) >> 1) * np + p) * 2 * kWarp + lane * 2 + ((R0 + r) & 1)];
  };
  auto bwd_at = [&](int64_t r, int p) -> double& {
    return P.shared ? F.bwd[r * 2 + p] : F.bwd[(((R0 + r) >> 1) * 2 + p) * 2 * kWarp + lane * 2 + ((R0 + r) & 1)];
  };
  int64_t r = 0;
  if (s >= 0) {
    const int64_t n = P.shared ? P.n_shared : P.n[s];
    const int64_t o = P.shared ? 0 : P.off[s];
    const double sg = sigma ? sigma[P.shared ? 0 : s] : 0.0;
    double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;  // gamma/delta of rows r-2, r-1
    for (; r < n; ++r) {
      double ar, br, cr, dr, er;
      if (sigma && r >= 2 && r + 2 < n) {  // interior rows of I + sigma D4: [1, -4, 6, -4, 1]
        ar = sg;
        br = -4.0 * sg;
        cr = 1.0 + sg * 6.0;
        dr = br;
        er = sg;
      } else if (sigma) {
        double w[5];
        d4_weights(r, n, w);
        ar = sg * w[0];
        br = sg * w[1];
        cr = 1.0 + sg * w[2];
        dr = sg * w[3];
        er = sg * w[4];
      } else {
        cr = c[o + r];
        ar = (r >= 2) ? a[o + r] : 0.0;
        br = (r >= 1) ? b[o + r] : 0.0;
        dr = (r + 1 < n) ? d[o + r] : 0.0;
        er = (r + 2 < n) ? e[o + r] : 0.0;
      }
      if (r < 2) ar = 0.0;
      if (r < 1) br = 0.0;
      if (r + 1 >= n) dr = 0.0;
      if (r + 2 >= n) er = 0.0;
      const double beta = br - ar * gam2;
      const double alpha = cr - ar * del2 - beta * gam1;
      if (!(alpha != 0.0) || !isfinite(alpha)) {
        report_bad_pivot(P.info, s, r);
        break;
      }
      // one reciprocal per row, then products (each FP64 division is several operations on the
      // 1/64-rate FP64 pipe)
      const double ia = 1.0 / alpha;
      const double gamma = (dr - beta * del1) * ia;
      const double delta = er * ia;
      fwd_at(r, 0) = ia;
      if (hyp) {
        fwd_at(r, 1) = beta;
      } else {
        fwd_at(r, 1) = beta * ia;
        fwd_at(r, 2) = ar * ia;
      }
      bwd_at(r, 0) = gamma;
      bwd_at(r, 1) = delta;
      gam2 = gam1;
      del2 = del1;
      gam1 = gamma;
      del1 = delta;
    }
  }
  for (; r < Lg; ++r) {
    fwd_at(r, 0) = hyp ? 0.0 : 1.0;
    fwd_at(r, 1) = 0.0;
    if (!hyp) fwd_at(r, 2) = 0.0;
    bwd_at(r, 0) = 0.0;
    bwd_at(r, 1) = 0.0;
  }
}

struct Lane {
  int64_t s;   // system index (-1 for an empty lane)
  int64_t n;   // rows of this lane's system (0 for an empty lane)
  int64_t fo;  // first row of the system in f/x
  int64_t Lg;  // rows walked by the warp
  int64_t R0;  // first record row of the warp
};

template <bool SHARED>
__device__ __forceinline__ Lane lane_setup(const DevPlan& P, int64_t k, int lane) {
  Lane L;
  const int64_t q = k * kWarp + lane;
  if (SHARED) {
    L.s = (q < P.batch) ? q : -1;
    L.n = (q < P.batch) ? P.n_shared : 0;
    L.fo = (q < P.batch) ? q * P.n_shared : 0;
    L.Lg = P.n_shared;
    L.R0 = k * P.n_shared;
  } else {
    const int s = P.perm[q];
    L.s = s;
    L.n = (s >= 0) ? P.n[s] : 0;
    L.fo = (s >= 0) ? P.off[s] : 0;
    L.Lg = P.glen[k];
    L.R0 = P.goff[k];
  }
  return L;
}

template <bool SHARED, int NP = 3>
__device__ __forceinline__ int64_t fwd_idx(const Lane& L, int64_t r, int p, int lane) {
  return SHARED ? r * 3 + p : (((L.R0 + r) >> 1) * NP + p) * 2 * kWarp + lane * 2 + ((L.R0 + r) & 1);
}
template <bool SHARED>
__device__ __forceinline__ int64_t bwd_idx(const Lane& L, int64_t r, int p, int lane) {
  return SHARED ? r * 2 + p : (((L.R0 + r) >> 1) * 2 + p) * 2 * kWarp + lane * 2 + ((L.R0 + r) & 1);
}
// Scratch row r of the lane (g of the forward sweep, z of the adjoint).
template <bool SHARED>
__device__ __forceinline__ int64_t scr_idx(const Lane& L, int64_t r, int lane) {
  return SHARED ? (L.R0 + r) * kWarp + lane : (((L.R0 + r) >> 1) * kWarp + lane) * 2 + ((L.R0 + r) & 1);
}

// The lane's interior records: pairs lo .. hi take them from registers (lo > hi: none).
struct Interior {
  double2 ia = {0.0, 0.0}, be = {0.0, 0.0}, ga = {0.0, 0.0}, de = {0.0, 0.0};
  int64_t lo = INT64_MAX, hi = -1;
};
__device__ __forceinline__ Interior interior_of(const F64Factors& F, const Lane& L, int64_t k, int lane) {
  Interior I;
  if (F.ik && L.s >= 0) {
    const int64_t q = k * kWarp + lane;
    const int K = F.ik[q];
    if (K != INT_MAX) {
      I.ia = F.icst[q * 4 + 0];
      I.be = F.icst[q * 4 + 1];
      I.ga = F.icst[q * 4 + 2];
      I.de = F.icst[q * 4 + 3];
      I.lo = K;
      I.hi = (L.n - 4) / 2;
    }
  }
  return I;
}

// x = A^{-1} f by the forward substitution L g = f and the back substitution
// R x = g (Sec. 2.4).  With the stored 1/alpha, beta/alpha, epsilon/alpha:
//   g_i = (1/alpha_i) f_i - (epsilon_i/alpha_i) g_{i-2} - (beta_i/alpha_i) g_{i-1}
//   x_i = g_i - gamma_i x_{i+1} - delta_i x_{i+2}
// g goes to the warp's scratch rows (coalesced) and comes back in reverse.
// Loads run U rows ahead of the arithmetic (register double buffering) so each
// lane keeps several independent memory requests in flight.
template <bool SHARED, int U>
__global__ void __launch_bounds__(256) k_solve64(DevPlan P, F64Factors F, const double* f, double* x,
                                                 double* __restrict__ gscr, int64_t kbeg, int64_t kend) {
  const int64_t k = kbeg + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (k >= kend) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const Lane L = lane_setup<SHARED>(P, k, lane);
  const double* __restrict__ fwd = F.fwd;
  const double* __restrict__ bwd = F.bwd;

  // ---- forward: L g = f ----
  double ca[U], cb[U], ce[U], cf[U];
  double na[U], nb[U], ne[U], nf[U];
  auto load_f = [&](int64_t r0, double* A, double* B, double* E, double* Fv) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = r0 + u;
      if (r < L.Lg) {
        A[u] = __ldg(fwd + fwd_idx<SHARED>(L, r, 0, lane));
        B[u] = __ldg(fwd + fwd_idx<SHARED>(L, r, 1, lane));
        E[u] = __ldg(fwd + fwd_idx<SHARED>(L, r, 2, lane));
        Fv[u] = (r < L.n) ? f[L.fo + r] : 0.0;
      }
    }
  };
  double g1 = 0.0, g2 = 0.0;
  load_f(0, ca, cb, ce, cf);
  for (int64_t r0 = 0; r0 < L.Lg; r0 += U) {
    if (r0 + U < L.Lg) load_f(r0 + U, na, nb, ne, nf);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = r0 + u;
      if (r < L.Lg) {
        const double g = fma(-cb[u], g1, fma(-ce[u], g2, ca[u] * cf[u]));
        gscr[scr_idx<SHARED>(L, r, lane)] = g;
        g2 = g1;
        g1 = g;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ca[u] = na[u];
      cb[u] = nb[u];
      ce[u] = ne[u];
      cf[u] = nf[u];
    }
  }

  // ---- back: R x = g ----
  double cg[U], cd[U], cG[U];
  double ng[U], nd[U], nG[U];
  auto load_b = [&](int64_t r0, double* Ga, double* De, double* Gv) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = r0 - u;
      if (r >= 0) {
        Ga[u] = __ldg(bwd + bwd_idx<SHARED>(L, r, 0, lane));
        De[u] = __ldg(bwd + bwd_idx<SHARED>(L, r, 1, lane));
        Gv[u] = gscr[scr_idx<SHARED>(L, r, lane)];
      }
    }
  };
  double x1 = 0.0, x2 = 0.0;
  load_b(L.Lg - 1, cg, cd, cG);
  for (int64_t r0 = L.Lg - 1; r0 >= 0; r0 -= U) {
    if (r0 - U >= 0) load_b(r0 - U, ng, nd, nG);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = r0 - u;
      if (r >= 0) {
        const double xv = fma(-cg[u], x1, fma(-cd[u], x2, cG[u]));
        if (r < L.n) x[L.fo + r] = xv;
        x2 = x1;
        x1 = xv;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cg[u] = ng[u];
      cd[u] = nd[u];
      cG[u] = nG[u];
    }
  }
}

// The same substitutions for per-system factors, walking row pairs: every
// factor plane, the scratch g and (when aligned) f and x move 16 bytes per lane
// per access.  Loads run U2 pairs ahead of the arithmetic (register double
// buffering).  HYP: hyperdiffusion records, g_i = (1/alpha_i)(f_i - beta_i
// g_{i-1} - sigma g_{i-2}) with sigma in a register -- one factor plane (8 bytes
// per row) less to read than the general form, for the same FP64 operations.
// SHARED: one matrix for the whole batch (general records fwd[r*3 + p], bwd[r*2 + p],
// loaded as broadcasts; the system length must be even so that row pairs do not
// straddle systems); f, x and g still move in row pairs.
template <int U2, bool HYP, bool SHARED = false>
__global__ void __launch_bounds__(128) k_solve64_pair(DevPlan P, F64Factors F, const double* f, double* x,
                                                      double* __restrict__ gscr, int64_t kbeg, int64_t kend) {
  const int64_t k = kbeg + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (k >= kend) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const Lane L = lane_setup<SHARED>(P, k, lane);
  const double* __restrict__ fwd1 = F.fwd;
  const double* __restrict__ bwd1 = F.bwd;
  const double2* __restrict__ fwd = reinterpret_cast<const double2*>(F.fwd);
  const double2* __restrict__ bwd = reinterpret_cast<const double2*>(F.bwd);
  double2* __restrict__ g2s = reinterpret_cast<double2*>(gscr);
  const int64_t np = L.Lg >> 1;   // pairs walked by the warp (Lg is even)
  const int64_t P0 = L.R0 >> 1;   // first record pair of the warp
  const bool fvec = ((L.fo & 1) == 0) && ((((uintptr_t)f) & 15) == 0);
  const bool xvec = ((L.fo & 1) == 0) && ((((uintptr_t)x) & 15) == 0);
  const double sg = (HYP && L.s >= 0) ? F.sig[L.s] : 0.0;
  constexpr int NP = HYP ? 2 : 3;
  const Interior I = (HYP && !SHARED) ? interior_of(F, L, k, lane) : Interior{};

  // ---- forward: L g = f ----
  double2 ca[U2], cb[U2], ce[U2], cf[U2];
  double2 na[U2], nb[U2], ne[U2], nf[U2];
  auto load_f = [&](int64_t q0, double2* A, double2* B, double2* E, double2* Fv) {
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 + u;
      if (q < np) {
        if (SHARED) {
          const double* ra = fwd1 + (2 * q) * 3;
          A[u] = make_double2(__ldg(ra), __ldg(ra + 3));
          B[u] = make_double2(__ldg(ra + 1), __ldg(ra + 4));
          E[u] = make_double2(__ldg(ra + 2), __ldg(ra + 5));
        } else if (HYP && q >= I.lo && q <= I.hi) {  // interior: the records are known
          A[u] = I.ia;
          B[u] = I.be;
        } else {
          const double2* rec = fwd + ((P0 + q) * NP) * kWarp + lane;
          A[u] = __ldg(rec);
          B[u] = __ldg(rec + kWarp);
          if (!HYP) E[u] = __ldg(rec + 2 * kWarp);
        }
        const int64_t r = 2 * q;
        if (fvec && r + 1 < L.n) {
          Fv[u] = *reinterpret_cast<const double2*>(f + L.fo + r);
        } else {
          Fv[u].x = (r < L.n) ? f[L.fo + r] : 0.0;
          Fv[u].y = (r + 1 < L.n) ? f[L.fo + r + 1] : 0.0;
        }
      }
    }
  };
  double g1 = 0.0, g2 = 0.0;
  load_f(0, ca, cb, ce, cf);
  for (int64_t q0 = 0; q0 < np; q0 += U2) {
    if (q0 + U2 < np) load_f(q0 + U2, na, nb, ne, nf);
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 + u;
      if (q < np) {
        double ga, gb;
        if (HYP) {
          ga = ca[u].x * fma(-cb[u].x, g1, fma(-sg, g2, cf[u].x));
          gb = ca[u].y * fma(-cb[u].y, ga, fma(-sg, g1, cf[u].y));
        } else {
          ga = fma(-cb[u].x, g1, fma(-ce[u].x, g2, ca[u].x * cf[u].x));
          gb = fma(-cb[u].y, ga, fma(-ce[u].y, g1, ca[u].y * cf[u].y));
        }
        g2s[(P0 + q) * kWarp + lane] = make_double2(ga, gb);
        g2 = ga;
        g1 = gb;
      }
    }
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      ca[u] = na[u];
      cb[u] = nb[u];
      ce[u] = ne[u];
      cf[u] = nf[u];
    }
  }

  // ---- back: R x = g ----
  double2 cg[U2], cd[U2], cG[U2];
  double2 ng[U2], nd[U2], nG[U2];
  auto load_b = [&](int64_t q0, double2* Ga, double2* De, double2* Gv) {
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 - u;
      if (q >= 0) {
        if (SHARED) {
          const double* rb = bwd1 + (2 * q) * 2;
          Ga[u] = make_double2(__ldg(rb), __ldg(rb + 2));
          De[u] = make_double2(__ldg(rb + 1), __ldg(rb + 3));
        } else if (HYP && q >= I.lo && q <= I.hi) {
          Ga[u] = I.ga;
          De[u] = I.de;
        } else {
          const double2* rec = bwd + ((P0 + q) * 2) * kWarp + lane;
          Ga[u] = __ldg(rec);
          De[u] = __ldg(rec + kWarp);
        }
        Gv[u] = g2s[(P0 + q) * kWarp + lane];
      }
    }
  };
  double x1 = 0.0, x2 = 0.0;
  load_b(np - 1, cg, cd, cG);
  for (int64_t q0 = np - 1; q0 >= 0; q0 -= U2) {
    if (q0 - U2 >= 0) load_b(q0 - U2, ng, nd, nG);
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 - u;
      if (q >= 0) {
        const double xb = fma(-cg[u].y, x1, fma(-cd[u].y, x2, cG[u].y));
        const double xa = fma(-cg[u].x, xb, fma(-cd[u].x, x1, cG[u].x));
        const int64_t r = 2 * q;
        if (xvec && r + 1 < L.n) {
          *reinterpret_cast<double2*>(x + L.fo + r) = make_double2(xa, xb);
        } else {
          if (r < L.n) x[L.fo + r] = xa;
          if (r + 1 < L.n) x[L.fo + r + 1] = xb;
        }
        x2 = xb;
        x1 = xa;
      }
    }
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      cg[u] = ng[u];
      cd[u] = nd[u];
      cG[u] = nG[u];
    }
  }
}

// ---- time steps with the right-hand side assembled in the solve ----
//
// One semi-implicit step per call on the field C (in place), for hyperdiffusion
// records (A_s = I + sigma_s D4, no-flux walls):
//   A_s C^{k+1} = f,  f_i = C_i + mu_s (D2 (C^3 - C))_i - nu_s (D4 C)_i,
// D2 and D4 the second and fourth differences with the same cell-centred
// reflection as the band (C_{-1} = C_0, C_{-2} = C_1, mirrored at the right).
// mu = D dt / dx^2, nu = 0 is the semi-implicit Cahn-Hilliard step of
// Sec. 2.1 (Eq. temporal) on the no-flux grid; mu = 0, nu = sigma gives a
// Crank-Nicolson step of Sec. 2.2 (Eq. 1d_hyper_scheme).  The forward sweep
// reads each C pair once, builds f from a window of three pairs and never
// stores it: the explicit part costs no memory traffic.

// f of rows base+2 and base+3 from v[k] = C_{base+k}, k = 0..5.
__device__ __forceinline__ void step_rhs_pair(const double (&v)[6], double mu, double nu, double& fa, double& fb) {
  fa = v[2];
  fb = v[3];
  if (nu != 0.0) {  // skipped for Cahn-Hilliard steps: the FP64 pipe is what bounds this kernel
    const double d4a = fma(6.0, v[2], fma(-4.0, v[1] + v[3], v[0] + v[4]));
    const double d4b = fma(6.0, v[3], fma(-4.0, v[2] + v[4], v[1] + v[5]));
    fa = fma(-nu, d4a, fa);
    fb = fma(-nu, d4b, fb);
  }
  if (mu != 0.0) {
    const double u1 = fma(v[1] * v[1], v[1], -v[1]), u2 = fma(v[2] * v[2], v[2], -v[2]);
    const double u3 = fma(v[3] * v[3], v[3], -v[3]), u4 = fma(v[4] * v[4], v[4], -v[4]);
    fa = fma(mu, fma(-2.0, u2, u1 + u3), fa);
    fb = fma(mu, fma(-2.0, u3, u2 + u4), fb);
  }
}

// Window v[k] = C_{2q-2+k} of a lane whose system has n rows, with the rows
// outside 0..n-1 replaced by their reflections (row n -> n-1, n+1 -> n-2,
// -1 -> 0, -2 -> 1; a one-row system is constant).  Rows past n+1 are only
// read for padding rows, whose f is discarded.
__device__ __forceinline__ void step_reflect(double (&v)[6], int64_t q, int64_t n) {
  const int64_t base = 2 * q - 2;
  if (n == 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = v[2];
    return;
  }
  if (base + 5 >= n) {
    double cn1 = 0.0, cn2 = 0.0;  // C_{n-1}, C_{n-2} (inside the window whenever a row < n needs them)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (base + k == n - 1) cn1 = v[k];
      if (base + k == n - 2) cn2 = v[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int64_t j = base + k;
      if (j >= n) v[k] = (j == n) ? cn1 : ((j == n + 1) ? cn2 : 0.0);
    }
  }
  if (q == 0) {
    v[0] = v[3];
    v[1] = v[2];
  }
}

template <int U2>
__global__ void __launch_bounds__(128) k_step64_pair(DevPlan P, F64Factors F, const double* __restrict__ mu_s,
                                                     const double* __restrict__ nu_s, double* C,
                                                     double* __restrict__ gscr, int64_t kbeg, int64_t kend) {
  const int64_t k = kbeg + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (k >= kend) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const Lane L = lane_setup<false>(P, k, lane);
  const double2* __restrict__ fwd = reinterpret_cast<const double2*>(F.fwd);
  const double2* __restrict__ bwd = reinterpret_cast<const double2*>(F.bwd);
  double2* __restrict__ g2s = reinterpret_cast<double2*>(gscr);
  const int64_t np = L.Lg >> 1;
  const int64_t P0 = L.R0 >> 1;
  const bool cvec = ((L.fo & 1) == 0) && ((((uintptr_t)C) & 15) == 0);
  const double sg = (L.s >= 0) ? F.sig[L.s] : 0.0;
  const double mu = (mu_s && L.s >= 0) ? mu_s[L.s] : 0.0;
  const double nu = (nu_s && L.s >= 0) ? nu_s[L.s] : 0.0;

  // ---- forward: L g = f, f assembled from C ----
  double2 ca[U2], cb[U2], cc[U2];
  double2 na[U2], nb[U2], nc[U2];
  auto load_f = [&](int64_t q0, double2* A, double2* B, double2* Cv) {
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 + u;
      A[u] = make_double2(0.0, 0.0);
      B[u] = A[u];
      Cv[u] = A[u];
      if (q < np) {
        const double2* rec = fwd + ((P0 + q) * 2) * kWarp + lane;
        A[u] = __ldg(rec);
        B[u] = __ldg(rec + kWarp);
        const int64_t r = 2 * q;
        if (cvec && r + 1 < L.n) {
          Cv[u] = *reinterpret_cast<const double2*>(C + L.fo + r);
        } else {
          Cv[u].x = (r < L.n) ? C[L.fo + r] : 0.0;
          Cv[u].y = (r + 1 < L.n) ? C[L.fo + r + 1] : 0.0;
        }
      }
    }
  };
  double g1 = 0.0, g2 = 0.0;
  double2 prev = make_double2(0.0, 0.0);  // C pair q - 1
  load_f(0, ca, cb, cc);
  for (int64_t q0 = 0; q0 < np; q0 += U2) {
    const bool more = q0 + U2 < np;
    if (more) load_f(q0 + U2, na, nb, nc);
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 + u;
      if (q < np) {
        const double2 nx = (u + 1 < U2) ? cc[u + 1] : (more ? nc[0] : make_double2(0.0, 0.0));
        double v[6] = {prev.x, prev.y, cc[u].x, cc[u].y, nx.x, nx.y};
        if (q == 0 || 2 * q + 3 >= L.n) step_reflect(v, q, L.n);
        double fa, fb;
        step_rhs_pair(v, mu, nu, fa, fb);
        if (2 * q >= L.n) fa = 0.0;
        if (2 * q + 1 >= L.n) fb = 0.0;
        const double ga = ca[u].x * fma(-cb[u].x, g1, fma(-sg, g2, fa));
        const double gb = ca[u].y * fma(-cb[u].y, ga, fma(-sg, g1, fb));
        g2s[(P0 + q) * kWarp + lane] = make_double2(ga, gb);
        g2 = ga;
        g1 = gb;
        prev = cc[u];
      }
    }
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      ca[u] = na[u];
      cb[u] = nb[u];
      cc[u] = nc[u];
    }
  }

  // ---- back: R x = g, x into C ----
  double2 cg[U2], cd[U2], cG[U2];
  double2 ng[U2], nd[U2], nG[U2];
  auto load_b = [&](int64_t q0, double2* Ga, double2* De, double2* Gv) {
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 - u;
      if (q >= 0) {
        const double2* rec = bwd + ((P0 + q) * 2) * kWarp + lane;
        Ga[u] = __ldg(rec);
        De[u] = __ldg(rec + kWarp);
        Gv[u] = g2s[(P0 + q) * kWarp + lane];
      }
    }
  };
  double x1 = 0.0, x2 = 0.0;
  load_b(np - 1, cg, cd, cG);
  for (int64_t q0 = np - 1; q0 >= 0; q0 -= U2) {
    if (q0 - U2 >= 0) load_b(q0 - U2, ng, nd, nG);
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = q0 - u;
      if (q >= 0) {
        const double xb = fma(-cg[u].y, x1, fma(-cd[u].y, x2, cG[u].y));
        const double xa = fma(-cg[u].x, xb, fma(-cd[u].x, x1, cG[u].x));
        const int64_t r = 2 * q;
        if (cvec && r + 1 < L.n) {
          *reinterpret_cast<double2*>(C + L.fo + r) = make_double2(xa, xb);
        } else {
          if (r < L.n) C[L.fo + r] = xa;
          if (r + 1 < L.n) C[L.fo + r + 1] = xb;
        }
        x2 = xb;
        x1 = xa;
      }
    }
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      cg[u] = ng[u];
      cd[u] = nd[u];
      cG[u] = nG[u];
    }
  }
}

// The same right-hand side written out (for the partitioned groups, whose
// chunked solve reads f from memory): one CTA per system of groups [kbeg, kend).
__global__ void __launch_bounds__(256) k_step_rhs(DevPlan P, const double* __restrict__ mu_s,
                                                  const double* __restrict__ nu_s, const double* __restrict__ C,
                                                  double* __restrict__ f, int64_t kbeg) {
  const int64_t q = kbeg * kWarp + blockIdx.x;
  const int32_t s = P.perm[q];
  if (s < 0) return;
  const int64_t n = P.n[s], o = P.off[s];
  const double mu = mu_s ? mu_s[s] : 0.0, nu = nu_s ? nu_s[s] : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      int64_t j = i + k - 2;
      while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
      v[k] = C[o + j];
    }
    double fi = v[2];
    if (nu != 0.0) fi = fma(-nu, fma(6.0, v[2], fma(-4.0, v[1] + v[3], v[0] + v[4])), fi);
    if (mu != 0.0) {
      const double u1 = fma(v[1] * v[1], v[1], -v[1]), u2 = fma(v[2] * v[2], v[2], -v[2]);
      const double u3 = fma(v[3] * v[3], v[3], -v[3]);
      fi = fma(mu, fma(-2.0, u2, u1 + u3), fi);
    }
    f[o + i] = fi;
  }
}

// ---- refactor and solve in one pass ----
//
// The paper's "Rewrite" use (Sec. 3): the matrix changes every call, so each
// call re-assembles A_s = I + sigma_s D4 from a new sigma_s and factors it
// (Sec. 2.4, factorisation steps) in the same sweep that runs the forward
// substitution, instead of a factor kernel followed by a solve that reads the
// factors back.  The records are still written (row pairs, hyperdiffusion
// form), so the plan is left factored with the new sigma for later solves.
__global__ void __launch_bounds__(128) k_refactor_solve64(DevPlan P, F64Factors F, const double* __restrict__ sigma,
                                                          const double* f, double* x, double* __restrict__ gscr,
                                                          int64_t kbeg, int64_t kend) {
  const int64_t k = kbeg + (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (k >= kend) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const Lane L = lane_setup<false>(P, k, lane);
  double2* __restrict__ fwd = reinterpret_cast<double2*>(F.fwd);
  double2* __restrict__ bwd = reinterpret_cast<double2*>(F.bwd);
  double2* __restrict__ g2s = reinterpret_cast<double2*>(gscr);
  double* __restrict__ sig = const_cast<double*>(F.sig);
  const int64_t np = L.Lg >> 1;
  const int64_t P0 = L.R0 >> 1;
  const bool fvec = ((L.fo & 1) == 0) && ((((uintptr_t)f) & 15) == 0);
  const bool xvec = ((L.fo & 1) == 0) && ((((uintptr_t)x) & 15) == 0);
  const double sg = (L.s >= 0) ? sigma[L.s] : 0.0;
  const double m4sg = -4.0 * sg, c6sg = 1.0 + sg * 6.0;
  if (L.s >= 0) sig[L.s] = sg;  // the plan's copy of sigma (epsilon of the records)

  // ---- factor + forward: L g = f ----
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;
  bool failed = L.s < 0;
  double g1 = 0.0, g2 = 0.0;
  for (int64_t q = 0; q < np; ++q) {
    double fv[2];
    const int64_t r0 = 2 * q;
    if (fvec && r0 + 1 < L.n) {
      const double2 t = *reinterpret_cast<const double2*>(f + L.fo + r0);
      fv[0] = t.x;
      fv[1] = t.y;
    } else {
      fv[0] = (r0 < L.n) ? f[L.fo + r0] : 0.0;
      fv[1] = (r0 + 1 < L.n) ? f[L.fo + r0 + 1] : 0.0;
    }
    double ia[2], bt[2], ga[2], de[2], gg[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = r0 + h;
      ia[h] = bt[h] = ga[h] = de[h] = 0.0;  // padding rows and rows after a failed pivot: g = x = 0
      if (r < L.n && !failed) {
        double ar = sg, br = m4sg, cr = c6sg, dr = m4sg, er = sg;  // interior rows: [1, -4, 6, -4, 1]
        if (r < 2 || r + 2 >= L.n) {                              // the two rows at each wall
          double w[5];
          d4_weights(r, L.n, w);
          ar = (r >= 2) ? sg * w[0] : 0.0;
          br = (r >= 1) ? sg * w[1] : 0.0;
          cr = 1.0 + sg * w[2];
          dr = (r + 1 < L.n) ? sg * w[3] : 0.0;
          er = (r + 2 < L.n) ? sg * w[4] : 0.0;
        }
        const double beta = br - ar * gam2;
        const double alpha = cr - ar * del2 - beta * gam1;
        if (!(alpha != 0.0) || !isfinite(alpha)) {
          report_bad_pivot(P.info, L.s, r);
          failed = true;
        } else {
          const double inv = 1.0 / alpha;
          ia[h] = inv;
          bt[h] = beta;
          ga[h] = (dr - beta * del1) * inv;
          de[h] = er * inv;
          gam2 = gam1;
          del2 = del1;
          gam1 = ga[h];
          del1 = de[h];
        }
      }
      // forward row in the hyperdiffusion form: g_i = (1/alpha_i)(f_i - beta_i g_{i-1} - sigma g_{i-2})
      gg[h] = ia[h] * fma(-bt[h], g1, fma(-sg, g2, fv[h]));
      g2 = g1;
      g1 = gg[h];
    }
    double2* rec = fwd + ((P0 + q) * 2) * kWarp + lane;
    rec[0] = make_double2(ia[0], ia[1]);
    rec[kWarp] = make_double2(bt[0], bt[1]);
    double2* rb = bwd + ((P0 + q) * 2) * kWarp + lane;
    rb[0] = make_double2(ga[0], ga[1]);
    rb[kWarp] = make_double2(de[0], de[1]);
    g2s[(P0 + q) * kWarp + lane] = make_double2(gg[0], gg[1]);
  }

  // ---- back: R x = g (records just written by this thread) ----
  double x1 = 0.0, x2 = 0.0;
  for (int64_t q = np - 1; q >= 0; --q) {
    const double2 G = bwd[((P0 + q) * 2) * kWarp + lane];
    const double2 D = bwd[((P0 + q) * 2 + 1) * kWarp + lane];
    const double2 Gv = g2s[(P0 + q) * kWarp + lane];
    const double xb = fma(-G.y, x1, fma(-D.y, x2, Gv.y));
    const double xa = fma(-G.x, xb, fma(-D.x, x1, Gv.x));
    const int64_t r = 2 * q;
    if (xvec && r + 1 < L.n) {
      *reinterpret_cast<double2*>(x + L.fo + r) = make_double2(xa, xb);
    } else {
      if (r < L.n) x[L.fo + r] = xa;
      if (r + 1 < L.n) x[L.fo + r + 1] = xb;
    }
    x2 = xb;
    x1 = xa;
  }
}

// ---- partitioned solve of groups of long systems ----
//
// A group's serial walk takes time proportional to its length however few of
// them there are, so groups of long systems are cut into chunks of kLongChunk
// rows and walked by one warp per (group, chunk).  The substitutions are
// second-order linear recurrences: a chunk maps the two values carried into
// it affinely, with a linear part that depends on the factors only (computed
// once per factorisation, k_cmaps64).  Pass 1 runs every chunk forward from a
// zero state; a scan per lane over the group's chunks gives the true entering
// states; pass 2 reruns the forward sweep (g to the scratch) and runs the back
// sweep from a zero state; a second scan; pass 3 reruns the back sweep (x).

struct PChunk {
  int64_t id;  // global chunk index
  int64_t k;   // group
  int64_t q0, q1;  // row pairs [q0, q1) of the chunk (relative to the group)
  bool active;
};

__device__ __forceinline__ PChunk pchunk(const DevPlan& P, const F64Part& X, int64_t c0, int64_t c1) {
  PChunk c;
  c.id = c0 + (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  c.active = c.id < c1;
  if (!c.active) return c;
  c.k = X.ck[c.id];
  const int64_t r0 = (int64_t)X.cc[c.id] * kLongChunk;
  c.q0 = r0 >> 1;
  c.q1 = min((int64_t)P.glen[c.k], r0 + kLongChunk) >> 1;
  return c;
}

// One forward row in either record form, and its homogeneous map on (g_{i-2}, g_{i-1}):
// g_i = -cE g_{i-2} - cB g_{i-1} + (inhomogeneous part).
template <bool HYP>
__device__ __forceinline__ double fwd_row(double a, double b, double e, double sg, double fv, double g1, double g2) {
  return HYP ? a * fma(-b, g1, fma(-sg, g2, fv)) : fma(-b, g1, fma(-e, g2, a * fv));
}

// Forward over the chunk's pairs from (g2, g1); WRITE stores g in the scratch.
template <bool HYP, bool WRITE>
__device__ __forceinline__ void pfwd(const Lane& L, const PChunk& c, const double2* __restrict__ fwd,
                                     const double* f, double2* __restrict__ g2s, double sg, bool fvec, int lane,
                                     double& g2, double& g1) {
  constexpr int NP = HYP ? 2 : 3;
  constexpr int B = 4;  // pairs loaded per batch
  const int64_t P0 = L.R0 >> 1;
  for (int64_t qb = c.q0; qb < c.q1; qb += B) {
    double2 A[B], Bv[B], Ev[B], Fv[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int64_t q = qb + u;
      if (q < c.q1) {
        const double2* rec = fwd + ((P0 + q) * NP) * kWarp + lane;
        A[u] = __ldg(rec);
        Bv[u] = __ldg(rec + kWarp);
        Ev[u] = HYP ? make_double2(0.0, 0.0) : __ldg(rec + 2 * kWarp);
        const int64_t r = 2 * q;
        if (fvec && r + 1 < L.n) {
          Fv[u] = *reinterpret_cast<const double2*>(f + L.fo + r);
        } else {
          Fv[u].x = (r < L.n) ? f[L.fo + r] : 0.0;
          Fv[u].y = (r + 1 < L.n) ? f[L.fo + r + 1] : 0.0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int64_t q = qb + u;
      if (q < c.q1) {
        const double ga = fwd_row<HYP>(A[u].x, Bv[u].x, Ev[u].x, sg, Fv[u].x, g1, g2);
        const double gb = fwd_row<HYP>(A[u].y, Bv[u].y, Ev[u].y, sg, Fv[u].y, ga, g1);
        if (WRITE) g2s[(P0 + q) * kWarp + lane] = make_double2(ga, gb);
        g2 = ga;
        g1 = gb;
      }
    }
  }
}

// Back over the chunk's pairs (descending) from (x1, x2) = (x_{r1}, x_{r1+1});
// WRITE stores x.
template <bool WRITE>
__device__ __forceinline__ void pbwd(const Lane& L, const PChunk& c, const double2* __restrict__ bwd,
                                     const double2* __restrict__ g2s, double* x, bool xvec, int lane, double& x1,
                                     double& x2) {
  constexpr int B = 4;
  const int64_t P0 = L.R0 >> 1;
  for (int64_t qb = c.q1 - 1; qb >= c.q0; qb -= B) {
    double2 G[B], D[B], Gv[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int64_t q = qb - u;
      if (q >= c.q0) {
        const double2* rec = bwd + ((P0 + q) * 2) * kWarp + lane;
        G[u] = __ldg(rec);
        D[u] = __ldg(rec + kWarp);
        Gv[u] = g2s[(P0 + q) * kWarp + lane];
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int64_t q = qb - u;
      if (q >= c.q0) {
        const double xb = fma(-G[u].y, x1, fma(-D[u].y, x2, Gv[u].y));
        const double xa = fma(-G[u].x, xb, fma(-D[u].x, x1, Gv[u].x));
        if (WRITE) {
          const int64_t r = 2 * q;
          if (xvec && r + 1 < L.n) {
            *reinterpret_cast<double2*>(x + L.fo + r) = make_double2(xa, xb);
          } else {
            if (r < L.n) x[L.fo + r] = xa;
            if (r + 1 < L.n) x[L.fo + r + 1] = xb;
          }
        }
        x2 = xb;
        x1 = xa;
      }
    }
  }
}

// Chunk maps from the records: forward on (g_{r0-2}, g_{r0-1}) -> (g_{r1-2}, g_{r1-1}),
// back on (x_{r1}, x_{r1+1}) -> (x_{r0}, x_{r0+1}); cmap[(id * 8 + e) * 32 + lane].
template <bool HYP>
__global__ void __launch_bounds__(256) k_cmaps64(DevPlan P, F64Factors F, F64Part X, int64_t c0, int64_t c1) {
  const PChunk c = pchunk(P, X, c0, c1);
  if (!c.active) return;
  const int lane = threadIdx.x;
  const Lane L = lane_setup<false>(P, c.k, lane);
  const double sg = (HYP && L.s >= 0) ? F.sig[L.s] : 0.0;
  constexpr int NP = HYP ? 2 : 3;
  const double2* fwd = reinterpret_cast<const double2*>(F.fwd);
  const double2* bwd = reinterpret_cast<const double2*>(F.bwd);
  const int64_t P0 = L.R0 >> 1;
  double f00 = 1.0, f01 = 0.0, f10 = 0.0, f11 = 1.0;
  for (int64_t q = c.q0; q < c.q1; ++q) {
    const double2* rec = fwd + ((P0 + q) * NP) * kWarp + lane;
    const double2 A = rec[0], Bv = rec[kWarp];
    const double2 Ev = HYP ? make_double2(0.0, 0.0) : rec[2 * kWarp];
    const double cB[2] = {HYP ? A.x * Bv.x : Bv.x, HYP ? A.y * Bv.y : Bv.y};
    const double cE[2] = {HYP ? A.x * sg : Ev.x, HYP ? A.y * sg : Ev.y};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double n10 = -cE[h] * f00 - cB[h] * f10, n11 = -cE[h] * f01 - cB[h] * f11;
      f00 = f10;
      f01 = f11;
      f10 = n10;
      f11 = n11;
    }
  }
  double b00 = 1.0, b01 = 0.0, b10 = 0.0, b11 = 1.0;
  for (int64_t q = c.q1 - 1; q >= c.q0; --q) {
    const double2* rec = bwd + ((P0 + q) * 2) * kWarp + lane;
    const double2 G = rec[0], D = rec[kWarp];
    const double gg[2] = {G.y, G.x}, dd[2] = {D.y, D.x};  // row 2q+1 first, then 2q
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double n00 = -gg[h] * b00 - dd[h] * b10, n01 = -gg[h] * b01 - dd[h] * b11;
      b10 = b00;
      b11 = b01;
      b00 = n00;
      b01 = n01;
    }
  }
  double* m = X.cmap + (c.id * 8) * kWarp + lane;
  m[0 * kWarp] = f00; m[1 * kWarp] = f01; m[2 * kWarp] = f10; m[3 * kWarp] = f11;
  m[4 * kWarp] = b00; m[5 * kWarp] = b01; m[6 * kWarp] = b10; m[7 * kWarp] = b11;
}

template <bool HYP>
__global__ void __launch_bounds__(256) k_pfwd0(DevPlan P, F64Factors F, F64Part X, const double* f, int64_t c0,
                                               int64_t c1) {
  const PChunk c = pchunk(P, X, c0, c1);
  if (!c.active) return;
  const int lane = threadIdx.x;
  const Lane L = lane_setup<false>(P, c.k, lane);
  const double sg = (HYP && L.s >= 0) ? F.sig[L.s] : 0.0;
  const bool fvec = ((L.fo & 1) == 0) && ((((uintptr_t)f) & 15) == 0);
  double g2 = 0.0, g1 = 0.0;
  pfwd<HYP, false>(L, c, reinterpret_cast<const double2*>(F.fwd), f, nullptr, sg, fvec, lane, g2, g1);
  X.U[c.id * kWarp + lane] = make_double2(g2, g1);
}

// Entering states of a group's chunks (thread per (group, lane)), in sweep order.
template <bool FWD>
__global__ void __launch_bounds__(256) k_pscan64(F64Part X, int64_t kbeg, int64_t kend) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = kbeg + t / kWarp;
  if (k >= kend) return;
  const int lane = (int)(t % kWarp);
  const int64_t base = X.cbase[k];
  const int nch = X.cnum[k];
  double e0 = 0.0, e1 = 0.0;
  for (int j = 0; j < nch; ++j) {
    const int64_t id = base + (FWD ? j : nch - 1 - j);
    X.E[id * kWarp + lane] = make_double2(e0, e1);
    const double* m = X.cmap + (id * 8 + (FWD ? 0 : 4)) * kWarp + lane;
    const double2 u = X.U[id * kWarp + lane];
    const double n0 = fma(m[0], e0, fma(m[kWarp], e1, u.x));
    const double n1 = fma(m[2 * kWarp], e0, fma(m[3 * kWarp], e1, u.y));
    e0 = n0;
    e1 = n1;
  }
}

template <bool HYP>
__global__ void __launch_bounds__(256) k_pmid(DevPlan P, F64Factors F, F64Part X, const double* f, double* gscr,
                                              int64_t c0, int64_t c1) {
  const PChunk c = pchunk(P, X, c0, c1);
  if (!c.active) return;
  const int lane = threadIdx.x;
  const Lane L = lane_setup<false>(P, c.k, lane);
  const double sg = (HYP && L.s >= 0) ? F.sig[L.s] : 0.0;
  const bool fvec = ((L.fo & 1) == 0) && ((((uintptr_t)f) & 15) == 0);
  double2* g2s = reinterpret_cast<double2*>(gscr);
  const double2 e = X.E[c.id * kWarp + lane];
  double g2 = e.x, g1 = e.y;
  pfwd<HYP, true>(L, c, reinterpret_cast<const double2*>(F.fwd), f, g2s, sg, fvec, lane, g2, g1);
  double x1 = 0.0, x2 = 0.0;
  pbwd<false>(L, c, reinterpret_cast<const double2*>(F.bwd), g2s, nullptr, false, lane, x1, x2);
  X.U[c.id * kWarp + lane] = make_double2(x1, x2);
}

__global__ void __launch_bounds__(256) k_pbwd(DevPlan P, F64Factors F, F64Part X, double* gscr, double* x,
                                              int64_t c0, int64_t c1) {
  const PChunk c = pchunk(P, X, c0, c1);
  if (!c.active) return;
  const int lane = threadIdx.x;
  const Lane L = lane_setup<false>(P, c.k, lane);
  const bool xvec = ((L.fo & 1) == 0) && ((((uintptr_t)x) & 15) == 0);
  const double2 e = X.E[c.id * kWarp + lane];
  double x1 = e.x, x2 = e.y;
  pbwd<true>(L, c, reinterpret_cast<const double2*>(F.bwd), reinterpret_cast<const double2*>(gscr), x, xvec, lane,
             x1, x2);
}

// y = A^{-T} f from the stored factors.  With L = D_alpha Lhat (Lhat unit lower
// with beta/alpha, epsilon/alpha) and A = L R:  A^T = R^T Lhat^T D_alpha, so
//   R^T z = f:      z_i = f_i - gamma_{i-1} z_{i-1} - delta_{i-2} z_{i-2}       (ascending)
//   Lhat^T w = z:   w_i = z_i - (beta/alpha)_{i+1} w_{i+1} - (eps/alpha)_{i+2} w_{i+2} (descending)
//   y_i = (1/alpha_i) w_i.
// Each sweep reads one record row per step; the couplings of later rows are
// carried in registers.
// HYP (hyperdiffusion records): (beta/alpha)_{i+1} = beta_{i+1} (1/alpha)_{i+1} and
// (eps/alpha)_{i+2} = sigma (1/alpha)_{i+2}, formed from the two stored planes.
template <bool SHARED, bool HYP>
__global__ void __launch_bounds__(256) k_adjoint64(DevPlan P, F64Factors F, const double* f, double* y,
                                                   double* __restrict__ zscr) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (k >= P.ngroups) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const Lane L = lane_setup<SHARED>(P, k, lane);
  const double* __restrict__ fwd = F.fwd;
  const double* __restrict__ bwd = F.bwd;
  // ascending: z
  double z1 = 0.0, z2 = 0.0;       // z_{i-1}, z_{i-2}
  double gam_m1 = 0.0, del_m1 = 0.0, del_m2 = 0.0;  // gamma_{i-1}, delta_{i-1}, delta_{i-2}
  for (int64_t r = 0; r < L.Lg; ++r) {
    const double fr = (r < L.n) ? f[L.fo + r] : 0.0;
    const double z = fma(-gam_m1, z1, fma(-del_m2, z2, fr));
    zscr[scr_idx<SHARED>(L, r, lane)] = z;
    z2 = z1;
    z1 = z;
    del_m2 = del_m1;
    gam_m1 = __ldg(bwd + bwd_idx<SHARED>(L, r, 0, lane));
    del_m1 = __ldg(bwd + bwd_idx<SHARED>(L, r, 1, lane));
  }
  // descending: w, y
  constexpr int NP = HYP ? 2 : 3;
  const double sg = (HYP && L.s >= 0) ? F.sig[L.s] : 0.0;
  double w1 = 0.0, w2 = 0.0;          // w_{i+1}, w_{i+2}
  double bp_p1 = 0.0, ep_p1 = 0.0, ep_p2 = 0.0;  // (beta/alpha)_{i+1}, (eps/alpha)_{i+1}, (eps/alpha)_{i+2}
  for (int64_t r = L.Lg - 1; r >= 0; --r) {
    const double ainv = __ldg(fwd + fwd_idx<SHARED, NP>(L, r, 0, lane));
    const double z = zscr[scr_idx<SHARED>(L, r, lane)];
    const double w = fma(-bp_p1, w1, fma(-ep_p2, w2, z));
    if (r < L.n) y[L.fo + r] = ainv * w;
    w2 = w1;
    w1 = w;
    ep_p2 = ep_p1;
    if (HYP) {
      bp_p1 = __ldg(fwd + fwd_idx<SHARED, NP>(L, r, 1, lane)) * ainv;
      ep_p1 = (r >= 2) ? sg * ainv : 0.0;
    } else {
      bp_p1 = __ldg(fwd + fwd_idx<SHARED, NP>(L, r, 1, lane));
      ep_p1 = __ldg(fwd + fwd_idx<SHARED, NP>(L, r, 2, lane));
    }
  }
}

// g_sigma[s] -= sum_i mu_i (D4 x)_i, one warp per system.
__global__ void k_sigma_grad(DevPlan P, const double* __restrict__ mu, const double* __restrict__ x,
                             double* g_sigma) {
  const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (s >= P.batch) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const int64_t n = P.shared ? P.n_shared : P.n[s];
  const int64_t o = P.shared ? s * P.n_shared : P.off[s];
  double acc = 0.0;
  for (int64_t i = lane; i < n; i += kWarp) {
    double d4x = 0.0;
    if (i >= 2 && i + 2 < n) {  // interior rows: [1, -4, 6, -4, 1], accumulated in the same order as below
      const double* xi = x + o + i;
      d4x = fma(-4.0, xi[-1], xi[-2]);
      d4x = fma(6.0, xi[0], d4x);
      d4x = fma(-4.0, xi[1], d4x);
      d4x = d4x + xi[2];
    } else {
      double w[5];
      d4_weights(i, n, w);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int64_t j = i + k - 2;
        if (j >= 0 && j < n && w[k] != 0.0) d4x = fma(w[k], x[o + j], d4x);
      }
    }
    acc = fma(mu[o + i], d4x, acc);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane == 0) g_sigma[s] -= acc;
}

inline int grid_for(int64_t threads, int block) { return (int)((threads + block - 1) / block); }

// ---- interior records of hyperdiffusion factorisations ----
//
// Rows 2 .. n - 3 of I + sigma D4 share one band row, and the factorisation's row step (Sec. 2.4)
// settles: past the first few dozen rows every row pair holds the same records bit for bit (a
// fixed point of the step, or a cycle of two rows, which row pairs also see as fixed).  The walks
// then take those records from registers instead of memory, with the same arithmetic.  One warp per
// group lane: ik = the first pair q of the run of pairs equal to pair (n - 4) / 2, the last pair whose
// rows are both interior (INT_MAX: n < 6), found by scanning back 32 pairs at a time; icst[4 q ..]
// = that pair's records (1/alpha, beta, gamma, delta), each a double2 of its two rows.
__global__ void k_interior64(DevPlan P, F64Factors F, double2* __restrict__ icst, int32_t* __restrict__ ik) {
  const int64_t qg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;  // group lane
  if (qg >= P.ngroups * kWarp) return;
  const int t = threadIdx.x & (kWarp - 1);
  const int lane = (int)(qg % kWarp);
  const Lane L = lane_setup<false>(P, qg / kWarp, lane);
  const double2* __restrict__ fwd = reinterpret_cast<const double2*>(F.fwd);
  const double2* __restrict__ bwd = reinterpret_cast<const double2*>(F.bwd);
  const int64_t P0 = L.R0 >> 1;
  auto same = [](double2 u, double2 v) {
    return __double_as_longlong(u.x) == __double_as_longlong(v.x) && __double_as_longlong(u.y) == __double_as_longlong(v.y);
  };
  int K = INT_MAX;
  double2 z[4] = {};
  const int64_t qe = (L.n - 4) / 2;
  if (L.s >= 0 && L.n >= 6) {
    z[0] = fwd[((P0 + qe) * 2 + 0) * kWarp + lane];
    z[1] = fwd[((P0 + qe) * 2 + 1) * kWarp + lane];
    z[2] = bwd[((P0 + qe) * 2 + 0) * kWarp + lane];
    z[3] = bwd[((P0 + qe) * 2 + 1) * kWarp + lane];
    K = 1;  // unless a pair differs
    for (int64_t base = qe; base >= 1; base -= kWarp) {
      const int64_t q = base - t;
      bool diff = false;
      if (q >= 1) {
        diff = !same(fwd[((P0 + q) * 2 + 0) * kWarp + lane], z[0]) || !same(fwd[((P0 + q) * 2 + 1) * kWarp + lane], z[1]) ||
               !same(bwd[((P0 + q) * 2 + 0) * kWarp + lane], z[2]) || !same(bwd[((P0 + q) * 2 + 1) * kWarp + lane], z[3]);
      }
      const unsigned m = __ballot_sync(0xffffffffu, diff);
      if (m) {  // the differing pair nearest the end is the one of the lowest thread with diff set
        K = (int)(base - (__ffs(m) - 1) + 1);
        break;
      }
    }
  }
  if (t == 0) {
    for (int p = 0; p < 4; ++p) icst[qg * 4 + p] = z[p];
    ik[qg] = K;
  }
}

// ---- windowed walks of groups of long hyperdiffusion systems ----
//
// A group whose rows are many times one window is walked as windows of its rows, one warp each,
// side by side: window (group k, first row w0, rows m, overlap O) runs the group's forward and
// back substitutions over rows w0 .. w0 + m - 1 only, entering each sweep with a zero state where
// it cuts the group (w0 > 0 for the forward sweep, w0 + m < Lg for the back sweep), and writes x
// only for the rows at least O from a cut.  The error a cut leaves decays as the powers of the
// interior row maps (forward (g_{i-2}, g_{i-1}) -> (g_{i-1}, g_i), back (x_{i+1}, x_{i+2}) ->
// (x_i, x_{i+1}), Sec. 2.4's recurrences with the interior factors); O is the fewest multiple of 8
// rows over which both shrink to 2^-56 for every system of the group, so the rows kept agree with
// the whole walk far below FP64 rounding.

constexpr double kWinTol64 = 1.3877787807814457e-17;  // 2^-56

// Overlap rows per group (k_overlap64): the group's largest over its systems of at least 8 rows,
// from the records of row n - 3 (interior), or 0x7fff if a system needs more than omax rows; and,
// if lover is not null, each system's own at its group lane (0 for systems under 8 rows).
__global__ void k_overlap64(DevPlan P, F64Factors F, int omax, int32_t* __restrict__ gover, int32_t* __restrict__ lover) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (k >= P.ngroups) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const Lane L = lane_setup<false>(P, k, lane);
  int O = 0;
  if (L.s >= 0 && L.n >= 8) {
    const int64_t r = L.n - 3;
    const double ia = F.fwd[fwd_idx<false, 2>(L, r, 0, lane)], be = F.fwd[fwd_idx<false, 2>(L, r, 1, lane)];
    const double ga = F.bwd[bwd_idx<false>(L, r, 0, lane)], de = F.bwd[bwd_idx<false>(L, r, 1, lane)];
    const double sg = F.sig[L.s];
    // P_f = M_f^j, P_b = M_b^j, one row at a time
    double fa = 1, fb = 0, fc = 0, fd = 1, ba = 1, bb = 0, bc = 0, bd = 1;
    O = 0x7fff;
    for (int j = 1; j <= omax; ++j) {
      const double na = fc, nb = fd, nc = -ia * (sg * fa + be * fc), nd = -ia * (sg * fb + be * fd);
      fa = na; fb = nb; fc = nc; fd = nd;
      const double ma = -ga * ba - de * bc, mb = -ga * bb - de * bd;
      bc = ba; bd = bb; ba = ma; bb = mb;
      const double nf = fmax(fmax(fabs(fa), fabs(fb)), fmax(fabs(fc), fabs(fd)));
      const double nbk = fmax(fmax(fabs(ba), fabs(bb)), fmax(fabs(bc), fabs(bd)));
      if (fmax(nf, nbk) <= kWinTol64) {
        O = (j + 7) / 8 * 8;
        break;
      }
    }
  }
  if (lover) lover[k * kWarp + lane] = O;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) O = max(O, __shfl_xor_sync(0xffffffffu, O, d));
  if (lane == 0) gover[k] = O;
}

// Overlap rows of f copied out before an in-place windowed walk: halo[w][side][pair][lane]
// (side 0: the O rows after a cut at w0, side 1: the O rows before a cut at w0 + m; rows past a
// system's end are zero), omax / 2 pairs a side.
__global__ void k_win64_halo(DevPlan P, const int4* __restrict__ win, int64_t nwin, int omax,
                             const double* __restrict__ f, double2* __restrict__ halo) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
  if (w >= nwin) return;
  const int lane = threadIdx.x & (kWarp - 1);
  const int4 d = win[w];
  const Lane L = lane_setup<false>(P, d.x, lane);
  const int w0 = d.y, m = d.z & 0xffff, O = d.z >> 16;
  const int hp = omax / 2;
  for (int side = 0; side < 2; ++side) {
    if (side == 0 ? w0 == 0 : w0 + m >= L.Lg) continue;
    const int64_t r0 = side == 0 ? w0 : w0 + m - O;
    double2* h = halo + ((w * 2 + side) * hp) * kWarp + lane;
    for (int q = 0; q < O / 2; ++q) {
      const int64_t r = r0 + 2 * q;
      h[q * kWarp] = make_double2(r < L.n ? f[L.fo + r] : 0.0, r + 1 < L.n ? f[L.fo + r + 1] : 0.0);
    }
  }
}

// The walk of one window (hyperdiffusion records, row pairs, U2 pairs of loads ahead), as
// k_solve64_pair.  g of the kept rows goes to the group's scratch rows (no other window keeps
// them), g of the O rows after them to the window's side scratch (side[w][pair][lane], omax / 2
// pairs), the rows before them need none.  halo: the overlap rows of f, or nullptr (read f).
// PERS: the persistent form, a resident grid whose warps take the windows in turn (else one
// warp per window).
// CTAs of 128 threads per SM the window walks' register allocation must allow (one-CTA-per-window
// forms of up to 2 row pairs in flight; more pairs would spill): 5 (96 registers a thread, a few
// spilled).  Uncapped (126 registers) the windows fill the SMs' register files and
// the shorter groups' walks, launched beside them, wait: on GB300 the uneven batch's FP64 step
// took 1.63-1.66 ms against 1.34-1.35 with the cap (6: 80 registers, more spills, 1.58 ms).
#ifndef PENT_W64_MIN_BLOCKS
#define PENT_W64_MIN_BLOCKS 5
#endif
template <int U2, bool PERS>
__global__ void __launch_bounds__(128, (PERS || U2 > 2) ? 1 : PENT_W64_MIN_BLOCKS) k_solve64w(DevPlan P, F64Factors F, const int4* __restrict__ win, int64_t nwin,
                                                  int omax, const double* f, double* x, double* __restrict__ gscr,
                                                  double2* __restrict__ side, const double2* __restrict__ halo) {
  const int64_t nwarps = PERS ? (int64_t)gridDim.x * blockDim.x / kWarp : nwin;
  const int lane = threadIdx.x & (kWarp - 1);
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp; w < nwin; w += nwarps) {
    const int4 d = win[w];
    const Lane L = lane_setup<false>(P, d.x, lane);
    const int w0 = d.y, m = d.z & 0xffff, O = d.z >> 16;
    const bool lcut = w0 > 0, rcut = w0 + m < L.Lg;
    const int hp = omax / 2, oh = O / 2;
    const int64_t q0 = w0 >> 1, q1 = (w0 + m) >> 1;                                    // pairs walked
    const int64_t k0 = (w0 + (lcut ? O : 0)) >> 1, k1 = (w0 + m - (rcut ? O : 0)) >> 1;  // pairs kept
    const double2* __restrict__ fwd = reinterpret_cast<const double2*>(F.fwd);
    const double2* __restrict__ bwd = reinterpret_cast<const double2*>(F.bwd);
    double2* __restrict__ g2s = reinterpret_cast<double2*>(gscr);
    double2* __restrict__ gside = side + (w * hp) * kWarp + lane;
    const double2* hl = halo ? halo + ((w * 2 + 0) * hp) * kWarp + lane : nullptr;
    const double2* hr = halo ? halo + ((w * 2 + 1) * hp) * kWarp + lane : nullptr;
    const int64_t P0 = L.R0 >> 1;
    // 16-byte accesses of f and x: a system starting at an even row reads and writes the pair
    // (2q, 2q + 1) as one double2; one starting at an odd row the aligned double2 (2q + 1, 2q + 2),
    // carrying row 2q from the previous one (forward) or row 2q + 2 in the state (back)
    const bool odd = (L.fo & 1) != 0;
    const bool fvec = ((((uintptr_t)f) & 15) == 0), xvec = ((((uintptr_t)x) & 15) == 0);
    const double sg = L.s >= 0 ? F.sig[L.s] : 0.0;
    const Interior I = interior_of(F, L, d.x, lane);
    double fcarry = 0.0;  // odd systems: f of row 2q for the next pair read from f
    bool cvalid = false;

    // ---- forward: L g = f over the window's pairs ----
    double2 ca[U2], cb[U2], cf[U2], na[U2], nb[U2], nf[U2];
    auto load_f = [&](int64_t qb, double2* A, double2* B, double2* Fv) {
#pragma unroll
      for (int u = 0; u < U2; ++u) {
        const int64_t q = qb + u;
        if (q < q1) {
          const int64_t r = 2 * q;
          if (q >= I.lo && q <= I.hi) {  // interior: the records are known
            A[u] = I.ia;
            B[u] = I.be;
          } else {
            const double2* rec = fwd + ((P0 + q) * 2) * kWarp + lane;
            A[u] = __ldg(rec);
            B[u] = __ldg(rec + kWarp);
          }
          if (hl && lcut && q < q0 + oh) {
            Fv[u] = hl[(q - q0) * kWarp];
            cvalid = false;
          } else if (hr && rcut && q >= q1 - oh) {
            Fv[u] = hr[(q - (q1 - oh)) * kWarp];
          } else if (fvec && !odd && r + 1 < L.n) {
            Fv[u] = *reinterpret_cast<const double2*>(f + L.fo + r);
          } else if (fvec && odd && r + 2 < L.n) {  // rows r + 1, r + 2 aligned; row r carried
            const double2 D = *reinterpret_cast<const double2*>(f + L.fo + r + 1);
            Fv[u] = make_double2(cvalid ? fcarry : f[L.fo + r], D.x);
            fcarry = D.y;
            cvalid = true;
          } else {
            Fv[u].x = (r < L.n) ? f[L.fo + r] : 0.0;
            Fv[u].y = (r + 1 < L.n) ? f[L.fo + r + 1] : 0.0;
            cvalid = false;
          }
        }
      }
    };
    double g1 = 0.0, g2 = 0.0;
    load_f(q0, ca, cb, cf);
    for (int64_t qb = q0; qb < q1; qb += U2) {
      if (qb + U2 < q1) load_f(qb + U2, na, nb, nf);
#pragma unroll
      for (int u = 0; u < U2; ++u) {
        const int64_t q = qb + u;
        if (q < q1) {
          const double ga = ca[u].x * fma(-cb[u].x, g1, fma(-sg, g2, cf[u].x));
          const double gb = ca[u].y * fma(-cb[u].y, ga, fma(-sg, g1, cf[u].y));
          if (q >= k1)
            gside[(q - k1) * kWarp] = make_double2(ga, gb);
          else if (q >= k0)
            g2s[(P0 + q) * kWarp + lane] = make_double2(ga, gb);
          g2 = ga;
          g1 = gb;
        }
      }
#pragma unroll
      for (int u = 0; u < U2; ++u) {
        ca[u] = na[u];
        cb[u] = nb[u];
        cf[u] = nf[u];
      }
    }

    // ---- back: R x = g from the window's end down to its first kept pair ----
    double2 cg[U2], cd[U2], cG[U2], ng[U2], nd[U2], nG[U2];
    auto load_b = [&](int64_t qb, double2* Ga, double2* De, double2* Gv) {
#pragma unroll
      for (int u = 0; u < U2; ++u) {
        const int64_t q = qb - u;
        if (q >= k0) {
          if (q >= I.lo && q <= I.hi) {
            Ga[u] = I.ga;
            De[u] = I.de;
          } else {
            const double2* rec = bwd + ((P0 + q) * 2) * kWarp + lane;
            Ga[u] = __ldg(rec);
            De[u] = __ldg(rec + kWarp);
          }
          Gv[u] = q >= k1 ? gside[(q - k1) * kWarp] : g2s[(P0 + q) * kWarp + lane];
        }
      }
    };
    double x1 = 0.0, x2 = 0.0;
    load_b(q1 - 1, cg, cd, cG);
    for (int64_t qb = q1 - 1; qb >= k0; qb -= U2) {
      if (qb - U2 >= k0) load_b(qb - U2, ng, nd, nG);
#pragma unroll
      for (int u = 0; u < U2; ++u) {
        const int64_t q = qb - u;
        if (q >= k0) {
          const double xb = fma(-cg[u].y, x1, fma(-cd[u].y, x2, cG[u].y));
          const double xa = fma(-cg[u].x, xb, fma(-cd[u].x, x1, cG[u].x));
          if (q < k1) {
            const int64_t r = 2 * q;
            if (!odd) {
              if (xvec && r + 1 < L.n) {
                *reinterpret_cast<double2*>(x + L.fo + r) = make_double2(xa, xb);
              } else {
                if (r < L.n) x[L.fo + r] = xa;
                if (r + 1 < L.n) x[L.fo + r + 1] = xb;
              }
            } else if (!xvec) {
              if (r < L.n) x[L.fo + r] = xa;
              if (r + 1 < L.n) x[L.fo + r + 1] = xb;
            } else {
              // rows r + 1 (this pair) and r + 2 (x1, the pair above, if kept) as one aligned double2;
              // row r goes out with the pair below, or alone at the window's first kept pair
              if (q + 1 < k1 && r + 2 < L.n) {
                *reinterpret_cast<double2*>(x + L.fo + r + 1) = make_double2(xb, x1);
              } else if (r + 1 < L.n) {
                x[L.fo + r + 1] = xb;
              }
              if (q == k0 && r < L.n) x[L.fo + r] = xa;
            }
          }
          x2 = xb;
          x1 = xa;
        }
      }
#pragma unroll
      for (int u = 0; u < U2; ++u) {
        cg[u] = ng[u];
        cd[u] = nd[u];
        cG[u] = nG[u];
      }
    }
  }
}


// ---- windowed walks, one window per thread (system windows) ----
//
// The same windows as above, but each thread walks one window of one system: window (group lane
// gl, first pair q0, kept pairs [k0, k1)) runs the system's forward substitution over pairs
// q0 .. q0 + Rp - 1 from a zero state (exact at q0 = 0) and, in a second launch, the back
// substitution from the window's last pair down to k0 from a zero state (exact where the window
// ends the system), writing x of the kept pairs only.  The forward step is written with one
// dependent operation a row (the products with g_{i-2} and f_i do not wait for g_{i-1}), so a
// window's serial chain is one FP64 operation a row in each sweep.  The overlap is the system's own (not the
// largest of its group), the windows are listed in the order of the caller's rows, so the 32
// threads of a warp read and write neighbouring rows of one or two systems, and the records are a
// per-system copy (sfwd / sbwd: pair q of the system at base + q, planes interleaved) made once
// per factorisation.  The forward launch has read every f before the back launch writes any x,
// so an in-place solve needs no copy of the overlap rows.
//
// Descriptor: int4 {gl, q0, k0, k1}; g of pair q (q >= k0) at gs[(w / 32) * Rp * 32 + (q - q0) * 32 + w % 32].
__device__ __forceinline__ Interior interior_of_gl(const F64Factors& F, int64_t gl, int64_t n) {
  Interior I;
  if (F.ik) {
    const int K = F.ik[gl];
    if (K != INT_MAX) {
      I.ia = F.icst[gl * 4 + 0];
      I.be = F.icst[gl * 4 + 1];
      I.ga = F.icst[gl * 4 + 2];
      I.de = F.icst[gl * 4 + 3];
      I.lo = K;
      I.hi = (n - 4) / 2;
    }
  }
  return I;
}

template <int U2>
__global__ void __launch_bounds__(128) k_swin64_fwd(DevPlan P, F64Factors F, const int4* __restrict__ win, int64_t nwin,
                                                    int Rp, const double2* __restrict__ sfwd,
                                                    const int64_t* __restrict__ sbase, const double* f,
                                                    double2* __restrict__ gs) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= nwin) return;
  const int4 d = win[w];
  const int s = P.perm[d.x];
  const int64_t n = P.n[s], fo = P.off[s];
  const int64_t q0 = d.y, k0 = d.z, q1 = min(q0 + (int64_t)Rp, (n + 1) >> 1);
  const double sg = F.sig[s];
  const Interior I = interior_of_gl(F, d.x, n);
  // the interior rows' 1/alpha, beta/alpha, sigma/alpha, formed as the record copy forms them
  const double2 iia = I.ia, iib = make_double2(I.ia.x * I.be.x, I.ia.y * I.be.y),
                iis = make_double2(I.ia.x * sg, I.ia.y * sg);
  const double2* __restrict__ rec = sfwd + 3 * sbase[d.x];
  double2* __restrict__ go = gs + (w >> 5) * (int64_t)Rp * kWarp + (w & (kWarp - 1));
  // 16-byte accesses of f: a system starting at an even row reads pair (2q, 2q + 1) as one
  // double2; one starting at an odd row reads the aligned double2s (2q - 1, 2q) and (2q + 1, 2q + 2)
  // of each pair (U2 + 1 of them for U2 pairs: no value is carried from one batch to the next)
  const bool odd = (fo & 1) != 0;
  const bool fvec = (((uintptr_t)f) & 15) == 0;
  auto ld_pair = [&](int64_t r) {  // rows r, r + 1 of the system (zero past its end)
    double2 v = make_double2(0.0, 0.0);
    if (fvec && r >= 0 && r + 1 < n) {
      v = *reinterpret_cast<const double2*>(f + fo + r);
    } else {
      if (r >= 0 && r < n) v.x = f[fo + r];
      if (r + 1 >= 0 && r + 1 < n) v.y = f[fo + r + 1];
    }
    return v;
  };
  double2 ca[U2], cb[U2], cc[U2], cf[U2], na[U2], nb[U2], nc[U2], nf[U2];
  auto load = [&](int64_t qb, double2* A, double2* B, double2* C, double2* Fv) {
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = qb + u;
      if (q < q1) {
        if (q >= I.lo && q <= I.hi) {
          A[u] = iia;
          B[u] = iib;
          C[u] = iis;
        } else {
          A[u] = __ldg(rec + 3 * q);
          B[u] = __ldg(rec + 3 * q + 1);
          C[u] = __ldg(rec + 3 * q + 2);
        }
      }
    }
    if (!odd) {
#pragma unroll
      for (int u = 0; u < U2; ++u)
        if (qb + u < q1) Fv[u] = ld_pair(2 * (qb + u));
    } else {
      double2 D[U2 + 1];
#pragma unroll
      for (int u = 0; u <= U2; ++u) D[u] = (qb + u <= q1) ? ld_pair(2 * (qb + u) - 1) : make_double2(0.0, 0.0);
#pragma unroll
      for (int u = 0; u < U2; ++u) Fv[u] = make_double2(D[u].y, D[u + 1].x);
    }
  };
  double g1 = 0.0, g2 = 0.0;
  load(q0, ca, cb, cc, cf);
  for (int64_t qb = q0; qb < q1; qb += U2) {
    if (qb + U2 < q1) load(qb + U2, na, nb, nc, nf);
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = qb + u;
      if (q < q1) {
        const double ga = fma(-cb[u].x, g1, fma(-cc[u].x, g2, ca[u].x * cf[u].x));
        const double gb = fma(-cb[u].y, ga, fma(-cc[u].y, g1, ca[u].y * cf[u].y));
        if (q >= k0) go[(q - q0) * kWarp] = make_double2(ga, gb);
        g2 = ga;
        g1 = gb;
      }
    }
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      ca[u] = na[u];
      cb[u] = nb[u];
      cc[u] = nc[u];
      cf[u] = nf[u];
    }
  }
}

template <int U2>
__global__ void __launch_bounds__(128) k_swin64_bwd(DevPlan P, F64Factors F, const int4* __restrict__ win, int64_t nwin,
                                                    int Rp, const double2* __restrict__ sbwd,
                                                    const int64_t* __restrict__ sbase, const double2* __restrict__ gs,
                                                    double* x) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= nwin) return;
  const int4 d = win[w];
  const int s = P.perm[d.x];
  const int64_t n = P.n[s], fo = P.off[s];
  const int64_t q0 = d.y, k0 = d.z, k1 = d.w, q1 = min(q0 + (int64_t)Rp, (n + 1) >> 1);
  const Interior I = interior_of_gl(F, d.x, n);
  const double2* __restrict__ rec = sbwd + 2 * sbase[d.x];
  const double2* __restrict__ gi = gs + (w >> 5) * (int64_t)Rp * kWarp + (w & (kWarp - 1));
  const bool odd = (fo & 1) != 0;
  const bool xvec = (((uintptr_t)x) & 15) == 0;
  double2 cg[U2], cd[U2], cG[U2], ng[U2], nd[U2], nG[U2];
  auto load = [&](int64_t qb, double2* Ga, double2* De, double2* Gv) {
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = qb - u;
      if (q >= k0) {
        if (q >= I.lo && q <= I.hi) {
          Ga[u] = I.ga;
          De[u] = I.de;
        } else {
          Ga[u] = __ldg(rec + 2 * q);
          De[u] = __ldg(rec + 2 * q + 1);
        }
        Gv[u] = gi[(q - q0) * kWarp];
      }
    }
  };
  double x1 = 0.0, x2 = 0.0;
  load(q1 - 1, cg, cd, cG);
  for (int64_t qb = q1 - 1; qb >= k0; qb -= U2) {
    if (qb - U2 >= k0) load(qb - U2, ng, nd, nG);
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      const int64_t q = qb - u;
      if (q >= k0) {
        const double xb = fma(-cg[u].y, x1, fma(-cd[u].y, x2, cG[u].y));
        const double xa = fma(-cg[u].x, xb, fma(-cd[u].x, x1, cG[u].x));
        if (q < k1) {
          const int64_t r = 2 * q;
          if (!odd && xvec && r + 1 < n) {
            *reinterpret_cast<double2*>(x + fo + r) = make_double2(xa, xb);
          } else if (!odd || !xvec) {
            if (r < n) x[fo + r] = xa;
            if (r + 1 < n) x[fo + r + 1] = xb;
          } else {
            // rows r + 1 (this pair) and r + 2 (x1, the pair above, if kept) as one aligned double2;
            // row r goes out with the pair below, or alone at the first kept pair
            if (q + 1 < k1 && r + 2 < n) {
              *reinterpret_cast<double2*>(x + fo + r + 1) = make_double2(xb, x1);
            } else if (r + 1 < n) {
              x[fo + r + 1] = xb;
            }
            if (q == k0 && r < n) x[fo + r] = xa;
          }
        }
        x2 = xb;
        x1 = xa;
      }
    }
#pragma unroll
    for (int u = 0; u < U2; ++u) {
      cg[u] = ng[u];
      cd[u] = nd[u];
      cG[u] = nG[u];
    }
  }
}

// Per-system copy of the records of the systems walked in system windows: warp (blockIdx.x,
// blockIdx.y) copies pairs [64 y, 64 y + 64) of windowed group wg[x] (and every gridDim.y * 64
// pairs after them), one lane per system (sbase[gl] < 0: none).  Forward, in the form whose row step has one dependent operation,
// g_i = (1/alpha_i) f_i - (beta_i / alpha_i) g_{i-1} - (sigma / alpha_i) g_{i-2}:
// sfwd[3 (base + q) + p] = 1/alpha, beta/alpha, sigma/alpha of pair q (p = 0, 1, 2, each the
// product of the record 1/alpha with beta or sigma); back, sbwd[2 (base + q) + p] = gamma, delta.
constexpr int kSrecPairs = 64;
__global__ void __launch_bounds__(32) k_srec64(DevPlan P, F64Factors F, const int32_t* __restrict__ wg,
                                               const int64_t* __restrict__ sbase, double2* __restrict__ sfwd,
                                               double2* __restrict__ sbwd) {
  const int64_t k = wg[blockIdx.x];
  const int lane = threadIdx.x;
  const Lane L = lane_setup<false>(P, k, lane);
  const int64_t gl = k * kWarp + lane;
  const int64_t b = L.s >= 0 ? sbase[gl] : -1;
  if (b < 0) return;
  const double2* __restrict__ fwd = reinterpret_cast<const double2*>(F.fwd);
  const double2* __restrict__ bwd = reinterpret_cast<const double2*>(F.bwd);
  const int64_t P0 = L.R0 >> 1, np = (L.n + 1) >> 1;
  const double sg = F.sig[L.s];
  for (int64_t qa = (int64_t)blockIdx.y * kSrecPairs; qa < np; qa += (int64_t)gridDim.y * kSrecPairs) {
    const int64_t qe = min(qa + (int64_t)kSrecPairs, np);
    for (int64_t q = qa; q < qe; ++q) {
      const double2 ia = fwd[((P0 + q) * 2) * kWarp + lane], be = fwd[((P0 + q) * 2 + 1) * kWarp + lane];
      sfwd[3 * (b + q)] = ia;
      sfwd[3 * (b + q) + 1] = make_double2(ia.x * be.x, ia.y * be.y);
      sfwd[3 * (b + q) + 2] = make_double2(ia.x * sg, ia.y * sg);
      sbwd[2 * (b + q)] = bwd[((P0 + q) * 2) * kWarp + lane];
      sbwd[2 * (b + q) + 1] = bwd[((P0 + q) * 2 + 1) * kWarp + lane];
    }
  }
}

}  // namespace

cudaError_t launch_factor64(const DevPlan& P, const double* a, const double* b, const double* c, const double* d,
                            const double* e, const double* sigma, F64Factors F, cudaStream_t st) {
  const int64_t nslots = P.shared ? 1 : P.ngroups * kWarp;
  const int block = 128;
  k_factor64<<<grid_for(nslots, block), block, 0, st>>>(P, a, b, c, d, e, sigma, F);
  return cudaGetLastError();
}

cudaError_t launch_solve64(const DevPlan& P, F64Factors F, const double* f, double* x, double* gscr, int block_warps,
                           int unroll, int64_t g0, int64_t g1, cudaStream_t st) {
  if (g1 <= g0) return cudaSuccess;
  const int block = kWarp * block_warps;
  const int grid = grid_for((g1 - g0) * kWarp, block);
  if (P.shared && (P.n_shared & 1) == 0) {  // row pairs of a shared matrix (even length)
#define PENT_U2S(U_, U2_)                                                               \
  if (unroll == U_) {                                                                   \
    k_solve64_pair<U2_, false, true><<<grid, block, 0, st>>>(P, F, f, x, gscr, g0, g1); \
    return cudaGetLastError();                                                          \
  }
    PENT_U2S(2, 1) PENT_U2S(4, 2) PENT_U2S(8, 4)
#undef PENT_U2S
    return cudaErrorInvalidValue;
  }
  if (P.shared) {
#define PENT_U(U_)                                                   \
  if (unroll == U_) {                                                \
    k_solve64<true, U_><<<grid, block, 0, st>>>(P, F, f, x, gscr, g0, g1); \
    return cudaGetLastError();                                       \
  }
    PENT_U(2) PENT_U(4) PENT_U(8)
#undef PENT_U
    return cudaErrorInvalidValue;
  }
  // per-system factors: row pairs, unroll rows = 2 x pairs ahead
  const bool hyp = F.sig != nullptr;
#define PENT_U2(U_, U2_)                                                       \
  if (unroll == U_) {                                                          \
    if (hyp)                                                                   \
      k_solve64_pair<U2_, true><<<grid, block, 0, st>>>(P, F, f, x, gscr, g0, g1);  \
    else                                                                             \
      k_solve64_pair<U2_, false><<<grid, block, 0, st>>>(P, F, f, x, gscr, g0, g1); \
    return cudaGetLastError();                                                 \
  }
  PENT_U2(2, 1) PENT_U2(4, 2) PENT_U2(8, 4)
#undef PENT_U2
  return cudaErrorInvalidValue;
}

cudaError_t launch_step64(const DevPlan& P, F64Factors F, const double* mu, const double* nu, double* C,
                          double* gscr, int block_warps, int unroll, int64_t g0, int64_t g1, cudaStream_t st) {
  if (g1 <= g0) return cudaSuccess;
  if (P.shared || !F.sig) return cudaErrorInvalidValue;
  const int block = kWarp * block_warps;
  const int grid = grid_for((g1 - g0) * kWarp, block);
  if (unroll == 2)
    k_step64_pair<1><<<grid, block, 0, st>>>(P, F, mu, nu, C, gscr, g0, g1);
  else if (unroll == 4)
    k_step64_pair<2><<<grid, block, 0, st>>>(P, F, mu, nu, C, gscr, g0, g1);
  else if (unroll == 8)
    k_step64_pair<4><<<grid, block, 0, st>>>(P, F, mu, nu, C, gscr, g0, g1);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_refactor_solve64(const DevPlan& P, F64Factors F, const double* sigma, const double* f, double* x,
                                    double* gscr, int block_warps, int64_t g0, int64_t g1, cudaStream_t st) {
  if (g1 <= g0) return cudaSuccess;
  if (P.shared || !F.sig) return cudaErrorInvalidValue;
  const int block = kWarp * block_warps;
  k_refactor_solve64<<<grid_for((g1 - g0) * kWarp, block), block, 0, st>>>(P, F, sigma, f, x, gscr, g0, g1);
  return cudaGetLastError();
}

cudaError_t launch_step_rhs(const DevPlan& P, const double* mu, const double* nu, const double* C, double* f,
                            int64_t g0, int64_t g1, cudaStream_t st) {
  if (g1 <= g0) return cudaSuccess;
  k_step_rhs<<<(unsigned)((g1 - g0) * kWarp), 256, 0, st>>>(P, mu, nu, C, f, g0);
  return cudaGetLastError();
}

cudaError_t launch_chunk_maps64(const DevPlan& P, F64Factors F, const F64Part& X, int64_t c0, int64_t c1,
                                cudaStream_t st) {
  if (c1 <= c0) return cudaSuccess;
  const dim3 blk(kWarp, 8);
  const unsigned grid = (unsigned)((c1 - c0 + 7) / 8);
  if (F.sig)
    k_cmaps64<true><<<grid, blk, 0, st>>>(P, F, X, c0, c1);
  else
    k_cmaps64<false><<<grid, blk, 0, st>>>(P, F, X, c0, c1);
  return cudaGetLastError();
}

cudaError_t launch_solve64_part(const DevPlan& P, F64Factors F, const F64Part& X, const double* f, double* x,
                                double* gscr, int64_t kbeg, int64_t kend, int64_t c0, int64_t c1, cudaStream_t st) {
  if (c1 <= c0) return cudaSuccess;
  const dim3 blk(kWarp, 8);
  const unsigned grid = (unsigned)((c1 - c0 + 7) / 8);
  const unsigned sgrid = (unsigned)grid_for((kend - kbeg) * kWarp, 256);
  if (F.sig) {
    k_pfwd0<true><<<grid, blk, 0, st>>>(P, F, X, f, c0, c1);
    k_pscan64<true><<<sgrid, 256, 0, st>>>(X, kbeg, kend);
    k_pmid<true><<<grid, blk, 0, st>>>(P, F, X, f, gscr, c0, c1);
  } else {
    k_pfwd0<false><<<grid, blk, 0, st>>>(P, F, X, f, c0, c1);
    k_pscan64<true><<<sgrid, 256, 0, st>>>(X, kbeg, kend);
    k_pmid<false><<<grid, blk, 0, st>>>(P, F, X, f, gscr, c0, c1);
  }
  k_pscan64<false><<<sgrid, 256, 0, st>>>(X, kbeg, kend);
  k_pbwd<<<grid, blk, 0, st>>>(P, F, X, gscr, x, c0, c1);
  return cudaGetLastError();
}

cudaError_t launch_adjoint64(const DevPlan& P, F64Factors F, const double* f, double* x, double* gscr,
                             int block_warps, cudaStream_t st) {
  const int block = kWarp * block_warps;
  const int grid = grid_for(P.ngroups * kWarp, block);
  if (P.shared)
    k_adjoint64<true, false><<<grid, block, 0, st>>>(P, F, f, x, gscr);
  else if (F.sig)
    k_adjoint64<false, true><<<grid, block, 0, st>>>(P, F, f, x, gscr);
  else
    k_adjoint64<false, false><<<grid, block, 0, st>>>(P, F, f, x, gscr);
  return cudaGetLastError();
}

cudaError_t launch_sigma_grad(const DevPlan& P, const double* mu, const double* x, double* g_sigma, cudaStream_t st) {
  const int block = 256;
  k_sigma_grad<<<grid_for(P.batch * kWarp, block), block, 0, st>>>(P, mu, x, g_sigma);
  return cudaGetLastError();
}

cudaError_t launch_overlap64(const DevPlan& P, F64Factors F, int omax, int32_t* gover, int32_t* lover, cudaStream_t st) {
  if (P.ngroups == 0 || P.shared || !F.sig) return cudaErrorInvalidValue;
  k_overlap64<<<grid_for(P.ngroups * kWarp, 128), 128, 0, st>>>(P, F, omax, gover, lover);
  return cudaGetLastError();
}

cudaError_t launch_srec64(const DevPlan& P, F64Factors F, const int32_t* wg, int64_t nwg, int64_t max_pairs,
                          const int64_t* sbase, double2* sfwd, double2* sbwd, cudaStream_t st) {
  if (nwg == 0) return cudaSuccess;
  if (P.shared || !F.sig || max_pairs <= 0) return cudaErrorInvalidValue;
  const int64_t ny = std::min<int64_t>((max_pairs + kSrecPairs - 1) / kSrecPairs, 65535);  // the CTAs loop beyond
  if (nwg > INT_MAX) return cudaErrorInvalidValue;
  k_srec64<<<dim3((unsigned)nwg, (unsigned)ny), kWarp, 0, st>>>(P, F, wg, sbase, sfwd, sbwd);
  return cudaGetLastError();
}

// Row pairs the back walks of system windows load ahead when the forward walks load 2 (unroll 4;
// 0: the same): 3, on GB300 the uneven FP64 step took 0.915 ms against 0.930 with 2 and 0.965
// with 4 (the back walk waits on its loads of g and the records more than the forward one).
#ifndef PENT_SWIN_BWD_U2
#define PENT_SWIN_BWD_U2 3
#endif
cudaError_t launch_swin64(const DevPlan& P, F64Factors F, const int4* win, int64_t nwin, int window_rows, int unroll,
                          int block_warps, const double2* sfwd, const double2* sbwd, const int64_t* sbase,
                          const double* f, double* x, double2* gs, cudaStream_t st) {
  if (nwin == 0) return cudaSuccess;
  if (P.shared || !F.sig || window_rows <= 0 || window_rows % 8 || block_warps < 1 || block_warps > 4)
    return cudaErrorInvalidValue;
  // one-warp CTAs by default: the windows' warps then spread over the SMs within one warp of each other
  const int Rp = window_rows / 2, block = kWarp * block_warps;
  const int grid = grid_for(nwin, block);
  auto go = [&](auto fk, auto bk) {
    fk<<<grid, block, 0, st>>>(P, F, win, nwin, Rp, sfwd, sbase, f, gs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bk<<<grid, block, 0, st>>>(P, F, win, nwin, Rp, sbwd, sbase, gs, x);
    return cudaGetLastError();
  };
#if PENT_SWIN_BWD_U2 == 4
  if (unroll == 4) return go(k_swin64_fwd<2>, k_swin64_bwd<4>);
#elif PENT_SWIN_BWD_U2 == 3
  if (unroll == 4) return go(k_swin64_fwd<2>, k_swin64_bwd<3>);
#endif
  if (unroll == 8) return go(k_swin64_fwd<4>, k_swin64_bwd<4>);
  if (unroll == 4) return go(k_swin64_fwd<2>, k_swin64_bwd<2>);
  if (unroll == 2) return go(k_swin64_fwd<1>, k_swin64_bwd<1>);
  return cudaErrorInvalidValue;
}

cudaError_t launch_solve64w(const DevPlan& P, F64Factors F, const int4* win, int64_t nwin, int omax, int unroll,
                            int block_warps, const double* f, double* x, double* gscr, double* side, double* halo,
                            bool persistent, cudaStream_t st) {
  if (nwin == 0) return cudaSuccess;
  if (P.shared || !F.sig || omax <= 0 || omax % 8 || block_warps < 1 || block_warps > 4) return cudaErrorInvalidValue;
  const int block = kWarp * block_warps;
  const int grid = grid_for(nwin * kWarp, block);
  double2* h = nullptr;
  if (f == x) {  // in place: the overlap rows are overwritten by the neighbouring windows
    h = reinterpret_cast<double2*>(halo);
    k_win64_halo<<<grid, block, 0, st>>>(P, win, nwin, omax, f, h);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  double2* sd = reinterpret_cast<double2*>(side);
  auto go = [&](auto kernel) {
    int g = grid;
    if (persistent) {  // as many CTAs as stay resident
      int dev = 0, sms = 0, per_sm = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
      if (e != cudaSuccess) return e;
      g = (int)std::min<int64_t>(grid, (int64_t)std::max(per_sm, 1) * sms);
    }
    kernel<<<g, block, 0, st>>>(P, F, win, nwin, omax, f, x, gscr, sd, h);
    return cudaGetLastError();
  };
  if (persistent) {
    if (unroll == 8) return go(k_solve64w<4, true>);
    if (unroll == 4) return go(k_solve64w<2, true>);
    if (unroll == 2) return go(k_solve64w<1, true>);
  } else {
    if (unroll == 8) return go(k_solve64w<4, false>);
    if (unroll == 4) return go(k_solve64w<2, false>);
    if (unroll == 2) return go(k_solve64w<1, false>);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_interior64(const DevPlan& P, F64Factors F, double2* icst, int32_t* ik, cudaStream_t st) {
  if (P.ngroups == 0 || P.shared || !F.sig) return cudaErrorInvalidValue;
  k_interior64<<<grid_for(P.ngroups * kWarp * kWarp, 128), 128, 0, st>>>(P, F, icst, ik);
  return cudaGetLastError();
}

}  // namespace pent
