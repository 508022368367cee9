// FP32 substitution with iterative refinement, one CTA per system.
//
// Why this shape.  On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, and
// conversions between FP64 and FP32 run on that same slow pipe.  The solve
// therefore runs entirely on the FP32 units: FP32 factors, FP32 substitutions,
// and a residual f - A x evaluated in double-FP32 ("float-float") arithmetic
// with error-free transformations (Knuth's two-sum, FMA-based two-product), so
// the refinement reaches FP64-level accuracy without FP64 instructions.  FP64
// inputs are split into float pairs and results reassembled with integer bit
// operations instead of conversion instructions.
//
// One CTA of P = 32 W threads -- or, for long systems, a thread-block cluster of
// C such CTAs on C SMs -- owns one system of n <= C P L rows: thread t holds
// rows t L .. t L + L - 1, their factors and their right-hand side in registers
// (all loaded with coalesced 16-byte accesses, since a thread's rows are
// contiguous).  Each substitution (Sec. 2.4: L g = f, then R x = g) is a
// second-order linear recurrence, so a thread's chunk acts on the two carried
// values as an affine map whose linear part depends on the factors only.  Once
// per launch the linear parts are composed by a Kogge-Stone shuffle scan in each
// warp and every level's window map is kept in shared memory (the "scan plan");
// each substitution then runs its chunk from a zero state for the affine part,
// scans only those two numbers with the stored window maps, carries them across
// warps and, in a cluster, across CTAs through distributed shared memory, and
// reruns the chunk from the true entering state.  The factors are read from HBM
// once per call and reused by every substitution of every refinement step.
//
// The hyperdiffusion matrices are symmetric, so A = L D^{-1} L^T with D the
// diagonal alpha of L: R = D^{-1} L^T, gamma_i = beta_{i+1} / alpha_i and
// delta_i = epsilon_{i+2} / alpha_i, and epsilon_i = a_i = sigma for every row
// i >= 2.  Only 1/alpha_i and beta_i are stored (8 bytes per row in FP32); the
// substitutions use them directly, g_i = (1/alpha_i)(v_i - beta_i g_{i-1} -
// sigma g_{i-2}) and x_i = g_i - (1/alpha_i)(beta_{i+1} x_{i+1} + sigma x_{i+2}).
#include <cooperative_groups.h>

#include <cmath>
#include <cstdint>

#include "ff.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace pent {
namespace {

using namespace ff;


// Coupling below this norm is dropped from the scans: it changes the carried
// values by less than FP32 resolution, and the refinement corrects the FP32
// solve anyway.
constexpr float kScanTol = 9.3132257e-10f;  // 2^-30
constexpr int kMaxLev = 5;                  // Kogge-Stone levels of a 32-lane warp

// Barrier over the CTA, or over the whole cluster when the system spans C > 1 CTAs.
__device__ __forceinline__ void csync(int C) {
  if (C > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
}

// A pointer into the shared memory of CTA `rank` of this cluster.
template <class T>
__device__ __forceinline__ T* remote(T* p, int rank) {
  return cg::this_cluster().map_shared_rank(p, rank);
}

// Maximum over the system's threads (CTA, or cluster).  sh: W + 1 slots.
template <class T>
__device__ __forceinline__ T system_max(T v, int lane, int warp, int W, int C, T* sh) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const T o = __shfl_xor_sync(0xffffffffu, v, d);
    v = v > o ? v : o;
  }
  if (W == 1 && C == 1) return v;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  T r = sh[0];
  for (int w = 1; w < W; ++w) r = r > sh[w] ? r : sh[w];
  if (C > 1) {
    if (threadIdx.x == 0) sh[W] = r;
    cg::this_cluster().sync();
    for (int k = 0; k < C; ++k) {
      const T q = remote(sh, k)[W];
      r = r > q ? r : q;
    }
  }
  return r;
}

// Shared scratch of one CTA (dynamic; W is a launch parameter).  The scan plan
// (win, pprev, wtot) is written once per launch; the per-scan slots (utot, red)
// rotate through four buffers, so one barrier per scan separates every write
// from the reads of the same buffer, in this CTA and in the other CTAs of a
// cluster.
struct SmemView {
  float4* win;    // [2][kMaxLev][P]: window map of every Kogge-Stone level (dir 0 forward, 1 back)
  float4* pprev;  // [2][P]: inclusive window map of the previous chunk in sweep order
  float4* wtot;   // [2][W + 1]: map of each warp's chunks, then of the whole CTA
  float4* edge;   // [P][2]: first two rows (hi, lo), last two rows (hi, lo)
  float2* utot;   // [4][W + 1]: affine parts of the warp and CTA maps of one scan
  float* red;     // [4][W + 1]
  int* redi;      // [W + 1]
  float* wrap;    // [16]: periodic systems: rows 0, 1, n-2, n-1 (hi, lo) for the wrap-around
                  // neighbours, then the tail of Navon's reduction (CTA 0's copy serves the cluster)
};

__host__ __device__ inline size_t smem_bytes(int W) {
  const size_t P = 32 * (size_t)W;
  return sizeof(float4) * (2 * kMaxLev * P + 2 * P + 2 * (W + 1) + 2 * P) + sizeof(float2) * 4 * (W + 1) +
         sizeof(float) * 4 * (W + 1) + sizeof(int) * (W + 1) + sizeof(float) * 16;
}

__device__ __forceinline__ SmemView smem_view(unsigned char* base, int W) {
  const int P = 32 * W;
  SmemView v;
  v.win = reinterpret_cast<float4*>(base);
  v.pprev = v.win + 2 * kMaxLev * P;
  v.wtot = v.pprev + 2 * P;
  v.edge = v.wtot + 2 * (W + 1);
  v.utot = reinterpret_cast<float2*>(v.edge + 2 * P);
  v.red = reinterpret_cast<float*>(v.utot + 4 * (W + 1));
  v.redi = reinterpret_cast<int*>(v.red + 4 * (W + 1));
  v.wrap = reinterpret_cast<float*>(v.redi + (W + 1));
  return v;
}

struct Ctx {
  int lane, warp, t, P, W, C, rank;
  int nlev[2];  // Kogge-Stone levels of the forward and the back scan (warp-uniform)
  int phase;
};

// Scan plan of one sweep direction from this chunk's map m: the window map of
// every Kogge-Stone level (the map of the 2^l chunks ending at this one, before
// level l composes it further), the inclusive map of the previous chunk and
// each warp's total map.  These depend on the factors only, so every scan of
// the launch reuses them and composes just the affine parts.  The levels stop
// once every window either reaches the warp's first chunk or composes to a
// negligible map (later levels would only add terms multiplied by it).
template <bool FWD>
__device__ __forceinline__ int scan_setup(float4 m, const Ctx& cx, const SmemView& sm) {
  const int dir = FWD ? 0 : 1;
  float4* win = sm.win + dir * kMaxLev * cx.P;
  int nlev = 0;
#pragma unroll 1
  for (int l = 0; l < kMaxLev; ++l) {
    const int d = 1 << l;
    const bool done = (FWD ? (cx.lane < d) : (cx.lane + d > 31)) || mnorm(m) < kScanTol;
    if (__all_sync(0xffffffffu, done)) break;
    win[l * cx.P + cx.t] = m;
    const float4 o = shfl4<FWD>(m, d);
    if (FWD ? (cx.lane >= d) : (cx.lane + d < 32)) m = mmul(m, o);
    nlev = l + 1;
  }
  sm.pprev[dir * cx.P + cx.t] = shfl4<FWD>(m, 1);  // not read by the warp's first chunk
  if (FWD ? (cx.lane == 31) : (cx.lane == 0)) sm.wtot[dir * (cx.W + 1) + cx.warp] = m;
  return nlev;
}

// The CTA's total maps (cluster launches): the warp maps composed in sweep order.
__device__ __forceinline__ void cta_total_maps(const Ctx& cx, const SmemView& sm) {
  for (int dir = 0; dir < 2; ++dir) {
    const float4* wt = sm.wtot + dir * (cx.W + 1);
    float4 tm = make_float4(1.f, 0.f, 0.f, 1.f);
    for (int k = 0; k < cx.W; ++k) tm = mmul(wt[dir == 0 ? k : cx.W - 1 - k], tm);
    sm.wtot[dir * (cx.W + 1) + cx.W] = tm;
  }
}

// State entering this thread's chunk for a sweep through the system's chunks
// (FWD: increasing thread order, else decreasing), given the affine part
// (u0, u1) of this chunk's map (its result from a zero entering state).  The
// system is entered with state 0.
template <bool FWD>
__device__ __forceinline__ void scan_entry(float u0, float u1, Ctx& cx, const SmemView& sm, float& e0, float& e1) {
  const int dir = FWD ? 0 : 1;
  const float4* win = sm.win + dir * kMaxLev * cx.P;
#pragma unroll 1
  for (int l = 0; l < cx.nlev[dir]; ++l) {
    const int d = 1 << l;
    const float o0 = shfl<FWD>(u0, d), o1 = shfl<FWD>(u1, d);
    if (FWD ? (cx.lane >= d) : (cx.lane + d < 32)) {
      const float4 w = win[l * cx.P + cx.t];
      u0 = fmaf(w.x, o0, fmaf(w.y, o1, u0));
      u1 = fmaf(w.z, o0, fmaf(w.w, o1, u1));
    }
  }
  const float p0 = shfl<FWD>(u0, 1), p1 = shfl<FWD>(u1, 1);  // inclusive result of the previous chunk
  float c0 = 0.f, c1 = 0.f;                                  // state entering this warp
  const int W = cx.W, C = cx.C;
  if (W > 1 || C > 1) {
    float2* ut = sm.utot + (cx.phase++ & 3) * (W + 1);
    const float4* wt = sm.wtot + dir * (W + 1);
    if (FWD ? (cx.lane == 31) : (cx.lane == 0)) ut[cx.warp] = make_float2(u0, u1);
    __syncthreads();
    if (C > 1) {
      if (cx.t == 0) {  // the CTA's total affine part, published for the other CTAs of the cluster
        float a0 = 0.f, a1 = 0.f;
        for (int k = 0; k < W; ++k) {
          const int w = FWD ? k : W - 1 - k;
          apply(wt[w], ut[w], a0, a1);
        }
        ut[W] = make_float2(a0, a1);
      }
      cg::this_cluster().sync();
      if (FWD) {
        for (int r = 0; r < cx.rank; ++r) apply(remote(wt, r)[W], remote(ut, r)[W], c0, c1);
      } else {
        for (int r = C - 1; r > cx.rank; --r) apply(remote(wt, r)[W], remote(ut, r)[W], c0, c1);
      }
    }
    if (FWD) {
      for (int w = 0; w < cx.warp; ++w) apply(wt[w], ut[w], c0, c1);
    } else {
      for (int w = W - 1; w > cx.warp; --w) apply(wt[w], ut[w], c0, c1);
    }
  }
  if (FWD ? (cx.lane == 0) : (cx.lane == 31)) {
    e0 = c0;
    e1 = c1;
  } else {
    const float4 m = sm.pprev[dir * cx.P + cx.t];
    e0 = fmaf(m.x, c0, fmaf(m.y, c1, p0));
    e1 = fmaf(m.z, c0, fmaf(m.w, c1, p1));
  }
}

// The thread's factors: 1/alpha and beta of its L rows and beta of the next
// chunk's first row.  The symmetric hyperdiffusion band gives the rest:
// epsilon_i = sigma (i >= 2), gamma_i = beta_{i+1} / alpha_i, delta_i = sigma /
// alpha_i (i + 2 < n); the walls need no special case because the system is
// entered with state 0 at both ends and padding rows carry 1/alpha = 0.
template <int L>
struct Fac {
  float A[L];   // 1/alpha_i
  float Bt[L];  // beta_i
  float bnext;  // beta of row t L + L
  float sg;     // sigma (FP32)
};

// Forward map of the chunk on (g_{i-2}, g_{i-1}): g_i = A_i (v_i - beta_i g_{i-1} - sigma g_{i-2}).
template <int L>
__device__ __forceinline__ float4 fwd_chunk_map(const Fac<L>& fc) {
  float4 F = make_float4(1.f, 0.f, 0.f, 1.f);
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float n0 = -fc.A[j] * fmaf(fc.sg, F.x, fc.Bt[j] * F.z);
    const float n1 = -fc.A[j] * fmaf(fc.sg, F.y, fc.Bt[j] * F.w);
    F = make_float4(F.z, F.w, n0, n1);
  }
  return F;
}

// Back map of the chunk on (x_{i+1}, x_{i+2}): x_i = g_i - A_i (beta_{i+1} x_{i+1} + sigma x_{i+2}).
template <int L>
__device__ __forceinline__ float4 bwd_chunk_map(const Fac<L>& fc) {
  float4 T = make_float4(1.f, 0.f, 0.f, 1.f);
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const float bn = (j + 1 < L) ? fc.Bt[j + 1] : fc.bnext;
    const float n0 = -fc.A[j] * fmaf(bn, T.x, fc.sg * T.z);
    const float n1 = -fc.A[j] * fmaf(bn, T.y, fc.sg * T.w);
    T = make_float4(n0, n1, T.x, T.y);
  }
  return T;
}

// In place v <- A^{-1} v (FP32): forward L g = v, then back R x = g (Sec. 2.4),
// each as a zero-state pass over the chunk, a scan for the entering state, and
// a second pass from it.
template <int L>
__device__ __forceinline__ void cta_solve32(float (&v)[L], const Fac<L>& fc, Ctx& cx, const SmemView& sm) {
  const float sg = fc.sg;
  float p2 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float g = fc.A[j] * fmaf(-fc.Bt[j], p1, fmaf(-sg, p2, v[j]));
    p2 = p1;
    p1 = g;
  }
  float e0, e1;
  scan_entry<true>(p2, p1, cx, sm, e0, e1);
  p2 = e0;
  p1 = e1;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float g = fc.A[j] * fmaf(-fc.Bt[j], p1, fmaf(-sg, p2, v[j]));
    v[j] = g;
    p2 = p1;
    p1 = g;
  }
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const float bn = (j + 1 < L) ? fc.Bt[j + 1] : fc.bnext;
    const float xv = fmaf(-fc.A[j], fmaf(bn, s1, sg * s2), v[j]);
    s2 = s1;
    s1 = xv;
  }
  scan_entry<false>(s1, s2, cx, sm, e0, e1);
  s1 = e0;
  s2 = e1;
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const float bn = (j + 1 < L) ? fc.Bt[j + 1] : fc.bnext;
    const float xv = fmaf(-fc.A[j], fmaf(bn, s1, sg * s2), v[j]);
    v[j] = xv;
    s2 = s1;
    s1 = xv;
  }
}


// previous chunk and the first two of the next, across warps through shared
// memory and across CTAs of a cluster through distributed shared memory.
__device__ __forceinline__ void exchange_edges(float4 own_first, float4 own_last, const Ctx& cx, const SmemView& sm,
                                               float4& prv, float4& nxt) {
  const int t = cx.t, P = cx.P;
  sm.edge[2 * t] = own_first;
  sm.edge[2 * t + 1] = own_last;
  csync(cx.C);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (t > 0)
    prv = sm.edge[2 * (t - 1) + 1];
  else
    prv = (cx.rank > 0) ? remote(sm.edge, cx.rank - 1)[2 * (P - 1) + 1] : zero;
  if (t + 1 < P)
    nxt = sm.edge[2 * (t + 1)];
  else
    nxt = (cx.rank + 1 < cx.C) ? remote(sm.edge, cx.rank + 1)[0] : zero;
}

// XL0: every xl is zero (the first refinement step), so the low parts drop out.
template <int L, bool XL0>
__device__ __forceinline__ void residual_ff(const float (&fh)[L], const float (&fl)[L], const float (&xh)[L],
                                            const float (&xl)[L], float (&r)[L], float sgh, float sgl, int n, int tg,
                                            const Ctx& cx, const SmemView& sm) {
  float4 prv, nxt;
  exchange_edges(make_float4(xh[0], xh[1], XL0 ? 0.f : xl[0], XL0 ? 0.f : xl[1]),
                 make_float4(xh[L - 2], xh[L - 1], XL0 ? 0.f : xl[L - 2], XL0 ? 0.f : xl[L - 1]), cx, sm, prv, nxt);
  // neighbour windows: rows tg L - 2 .. tg L + L + 1
  float wh[L + 4], wl[L + 4];
  wh[0] = prv.x;
  wh[1] = prv.y;
  wh[L + 2] = nxt.x;
  wh[L + 3] = nxt.y;
  wl[0] = prv.z;
  wl[1] = prv.w;
  wl[L + 2] = nxt.z;
  wl[L + 3] = nxt.w;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    wh[j + 2] = xh[j];
    wl[j + 2] = XL0 ? 0.f : xl[j];
  }
  fill_ghosts<L>(wh, tg, n);
  if (!XL0) fill_ghosts<L>(wl, tg, n);
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float res = XL0 ? residual_row(wh[j], 0.f, wh[j + 1], 0.f, wh[j + 2], 0.f, wh[j + 3], 0.f, wh[j + 4], 0.f,
                                         fh[j], fl[j], sgh, sgl)
                          : residual_row(wh[j], wl[j], wh[j + 1], wl[j + 1], wh[j + 2], wl[j + 2], wh[j + 3],
                                         wl[j + 3], wh[j + 4], wl[j + 4], fh[j], fl[j], sgh, sgl);
    r[j] = (tg * L + j < n) ? res : 0.f;  // padding rows past the end of the system
  }
}

// The same residual in native FP64 (the literal reading: FP64 band from sigma,
// FP64 x and f).  xd holds x in FP64 (scaled by 2^-kshift like f).  The edge
// slots carry the neighbouring rows as double pairs.
template <int L>
__device__ __forceinline__ void residual_f64(const double (&fd)[L], const double (&xd)[L], float (&r)[L], double sg,
                                             int n, int tg, const Ctx& cx, const SmemView& sm) {
  float4 pf4, nf4;
  const double2 f2 = make_double2(xd[0], xd[1]), l2 = make_double2(xd[L - 2], xd[L - 1]);
  exchange_edges(*reinterpret_cast<const float4*>(&f2), *reinterpret_cast<const float4*>(&l2), cx, sm, pf4, nf4);
  const double2 prv = *reinterpret_cast<const double2*>(&pf4);
  const double2 nxt = *reinterpret_cast<const double2*>(&nf4);
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int i = tg * L + j;
    const double a = (j >= 2) ? xd[j - 2] : (j == 1 ? prv.y : prv.x);
    const double b = (j >= 1) ? xd[j - 1] : prv.y;
    const double d = (j + 1 < L) ? xd[j + 1] : nxt.x;
    const double e = (j + 2 < L) ? xd[j + 2] : (j + 1 < L ? nxt.x : nxt.y);
    double y;
    if (i >= n) {  // padding row past the end of the system
      y = 0.0;
    } else if (i >= 2 && i + 2 < n) {
      y = fma(6.0, xd[j], fma(-4.0, b + d, a + e));
    } else {
      float w[5];
      d4_weights_f(i, n, w);
      y = (double)w[0] * a + (double)w[1] * b + (double)w[2] * xd[j] + (double)w[3] * d + (double)w[4] * e;
    }
    const double rr = fma(-sg, y, fd[j] - xd[j]);
    r[j] = (i < n) ? __double2float_rn(rr) : 0.f;
  }
}

// ---------------------------------------------------------------- periodic systems (Sec. 2.3)
//
// Row r of a periodic system of n rows (n >= 5) lives in thread r / L of the
// system, slot r % L.  The rows that wrap around -- 0 and 1 after row n - 1,
// n - 2 and n - 1 before row 0 -- are published by their owners into CTA 0's
// `wrap` slots before an exchange's barrier and read after it.

__device__ __forceinline__ float* wrap_slots(const Ctx& cx, const SmemView& sm) {
  return cx.C > 1 ? remote(sm.wrap, 0) : sm.wrap;
}

// Owners of rows 0, 1, n-2, n-1 write (hi, lo) to slots 0..7.
template <int L>
__device__ __forceinline__ void publish_wrap(const float (&h)[L], const float (&l)[L], int tg, int n, float* slots) {
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int r = tg * L + j;
    const int k = (r == 0) ? 0 : (r == 1) ? 1 : (r == n - 2) ? 2 : (r == n - 1) ? 3 : -1;
    if (k >= 0) {
      slots[2 * k] = h[j];
      slots[2 * k + 1] = l[j];
    }
  }
}

// Window w[0 .. L+3] holds rows tg L - 2 .. tg L + L + 1; put the wrapped rows in
// (rows -2, -1 are n-2, n-1; rows n, n+1 are 0, 1).  Rows past n + 1 only feed
// padding rows.
template <int L>
__device__ __forceinline__ void fill_wrap(float (&wh)[L + 4], float (&wl)[L + 4], int tg, int n, const float* slots) {
  if (tg == 0) {
    wh[0] = slots[4];
    wl[0] = slots[5];
    wh[1] = slots[6];
    wl[1] = slots[7];
  }
#pragma unroll
  for (int q = 2; q < L + 4; ++q) {
    const int r = tg * L + q - 2;
    if (r == n) {
      wh[q] = slots[0];
      wl[q] = slots[1];
    } else if (r == n + 1) {
      wh[q] = slots[2];
      wl[q] = slots[3];
    }
  }
}

// Navon's reduction around the FP32 solve of E (the first m = n - 2 rows; rows
// m, m+1 are padding of the factorisation).  The periodic hyperdiffusion matrix
// is symmetric, so h = k and E^{-1} k = Z (stored per row): with y = E^{-1} f-hat
// from the plain solve, Eq. (first_two) gives t = S^{-1} (f_tail - h^T y), where
// h^T y needs only y_0, y_1, y_{m-2}, y_{m-1}, and Eq. (solve) gives
// x = E^{-1} (f-hat - k t) = y - Z t.  periodic_tail_rhs publishes f_m, f_{m+1}
// before the solve; periodic_tail finishes after it.
template <int L>
__device__ __forceinline__ void periodic_tail_rhs(const float (&v)[L], int tg, int n, const Ctx& cx,
                                                  const SmemView& sm) {
  float* slots = wrap_slots(cx, sm) + 8;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int r = tg * L + j;
    if (r == n - 2) slots[4] = v[j];
    if (r == n - 1) slots[5] = v[j];
  }
}

template <int L, int NPL>
__device__ __forceinline__ void periodic_tail(float (&v)[L], const float4* __restrict__ gq, int PT, int tg, int n,
                                              float sg, float4 si, const Ctx& cx, const SmemView& sm) {
  const int m = n - 2;
  float* slots = wrap_slots(cx, sm) + 8;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int r = tg * L + j;
    if (r == 0) slots[0] = v[j];
    if (r == 1) slots[1] = v[j];
    if (r == m - 2) slots[2] = v[j];
    if (r == m - 1) slots[3] = v[j];
  }
  csync(cx.C);
  const float y0 = slots[0], y1 = slots[1], ym2 = slots[2], ym1 = slots[3], fa = slots[4], fb = slots[5];
  // rows n-2 and n-1 of A restricted to E's columns: (sigma @ 0, sigma @ m-2, -4 sigma @ m-1) and
  // (-4 sigma @ 0, sigma @ 1, sigma @ m-1)
  const float r0 = fa - sg * fmaf(-4.f, ym1, y0 + ym2);
  const float r1 = fb - sg * fmaf(-4.f, y0, y1 + ym1);
  const float t0 = fmaf(si.x, r0, si.y * r1), t1 = fmaf(si.z, r0, si.w * r1);
#pragma unroll
  for (int jq = 0; jq < L / 4; ++jq) {
    const float4 za = __ldg(gq + (int64_t)(jq * NPL + 2) * PT + tg), zb = __ldg(gq + (int64_t)(jq * NPL + 3) * PT + tg);
    const float z0[4] = {za.x, za.y, za.z, za.w}, z1[4] = {zb.x, zb.y, zb.z, zb.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * jq + u, r = tg * L + j;
      v[j] = (r < m) ? fmaf(-z0[u], t0, fmaf(-z1[u], t1, v[j])) : (r == m) ? t0 : (r == m + 1) ? t1 : 0.f;
    }
  }
}

// r = f - A x for a periodic system, in float-float (the stencil of
// residual_row with wrapped neighbours).
template <int L, bool XL0>
__device__ __forceinline__ void residual_ff_per(const float (&fh)[L], const float (&fl)[L], const float (&xh)[L],
                                                const float (&xl)[L], float (&r)[L], float sgh, float sgl, int n,
                                                int tg, const Ctx& cx, const SmemView& sm) {
  float zl[L];
#pragma unroll
  for (int j = 0; j < L; ++j) zl[j] = XL0 ? 0.f : xl[j];
  publish_wrap<L>(xh, zl, tg, n, wrap_slots(cx, sm));
  float4 prv, nxt;
  exchange_edges(make_float4(xh[0], xh[1], zl[0], zl[1]), make_float4(xh[L - 2], xh[L - 1], zl[L - 2], zl[L - 1]),
                 cx, sm, prv, nxt);
  float wh[L + 4], wl[L + 4];
  wh[0] = prv.x;
  wh[1] = prv.y;
  wh[L + 2] = nxt.x;
  wh[L + 3] = nxt.y;
  wl[0] = prv.z;
  wl[1] = prv.w;
  wl[L + 2] = nxt.z;
  wl[L + 3] = nxt.w;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    wh[j + 2] = xh[j];
    wl[j + 2] = zl[j];
  }
  fill_wrap<L>(wh, wl, tg, n, wrap_slots(cx, sm));
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float res = residual_row(wh[j], wl[j], wh[j + 1], wl[j + 1], wh[j + 2], wl[j + 2], wh[j + 3], wl[j + 3],
                                   wh[j + 4], wl[j + 4], fh[j], fl[j], sgh, sgl);
    r[j] = (tg * L + j < n) ? res : 0.f;
  }
}

// ---------------------------------------------------------------- explicit part of a time step (float-float)

// C^3 - C for C = ch + cl (float-float; cl^2 is below the pair's resolution and dropped).
__device__ __forceinline__ void cube_minus_ff(float ch, float cl, float& uh, float& ul) {
  float p, e, c2h, c2l, c3h, c3l;
  two_prod(ch, ch, p, e);
  e = fmaf(2.f * ch, cl, e);
  fast_two_sum(p, e, c2h, c2l);
  two_prod(c2h, ch, p, e);
  e = fmaf(c2h, cl, fmaf(c2l, ch, e));
  fast_two_sum(p, e, c3h, c3l);
  float s, es;
  two_sum(c3h, -ch, s, es);
  es = es + (c3l - cl);
  fast_two_sum(s, es, uh, ul);
}

// a + b - 2 c for float-float a, b, c (the second difference).
__device__ __forceinline__ void d2_ff(float ah, float al, float bh, float bl, float ch, float cl, float& dh,
                                      float& dl) {
  float s, e, t, e2;
  two_sum(ah, bh, s, e);
  e = e + (al + bl);
  two_sum(s, -2.f * ch, t, e2);  // 2 c is exact
  e = e + fmaf(-2.f, cl, e2);
  fast_two_sum(t, e, dh, dl);
}

// [1, -4, 6, -4, 1] applied to the float-float window a..e (the fourth difference).
__device__ __forceinline__ void d4_ff(float ah, float al, float bh, float bl, float ch, float cl, float dh, float dl,
                                      float eh, float el, float& yh, float& yl) {
  float s1, e1, s2, e2, t, e3, p, e4, S, Er;
  two_sum(ah, eh, s1, e1);
  two_sum(bh, dh, s2, e2);
  two_sum(s1, -4.f * s2, t, e3);
  two_prod(6.f, ch, p, e4);
  two_sum(t, p, S, Er);
  const float low = fmaf(6.f, cl, fmaf(-4.f, bl + dl, al + el));
  Er = Er + ((e1 - 4.f * e2) + (e3 + e4) + low);
  fast_two_sum(S, Er, yh, yl);
}

// (ph + pl) * (qh + ql) in float-float.
__device__ __forceinline__ void mul_ff(float ph, float pl, float qh, float ql, float& rh, float& rl) {
  float p, e;
  two_prod(ph, qh, p, e);
  e = fmaf(ph, ql, fmaf(pl, qh, e));
  fast_two_sum(p, e, rh, rl);
}

// The right-hand side of a semi-implicit step, f = C + mu D2(C^3 - C) - nu D4 C
// (Sec. 2.1, Eq. temporal; Sec. 2.2, Eq. 1d_hyper_scheme), for this thread's L
// rows from the field C in cv (FP64, unscaled), in float-float: each C is split
// into a float pair, the two rows on either side come from the neighbouring
// threads (and CTAs of a cluster), the no-flux walls mirror them, and the cube,
// the differences and the products are error-free transformations.  Rows past
// the end of the system get f = 0.
// twice: the Crank-Nicolson form with nu = sigma of the matrix, where
// A C' = C - sigma D4 C = 2 C - A C: the right-hand side is 2 C + mu D2(C^3 - C)
// (no cancellation) and the caller subtracts C from the solution.
template <int L, bool PER = false>
__device__ __forceinline__ void step_rhs_ff(const double (&cv)[L], float muh, float mul, float nuh, float nul,
                                            bool has_mu, bool has_nu, bool twice, float (&fh)[L], float (&fl)[L],
                                            int n, int tg, const Ctx& cx, const SmemView& sm) {
  float ch[L], cl[L];
#pragma unroll
  for (int j = 0; j < L; ++j) split_scaled(cv[j], 0, ch[j], cl[j]);
  if (PER) publish_wrap<L>(ch, cl, tg, n, wrap_slots(cx, sm));
  float4 prv, nxt;
  exchange_edges(make_float4(ch[0], ch[1], cl[0], cl[1]), make_float4(ch[L - 2], ch[L - 1], cl[L - 2], cl[L - 1]),
                 cx, sm, prv, nxt);
  float wh[L + 4], wl[L + 4];  // rows tg L - 2 .. tg L + L + 1
  wh[0] = prv.x;
  wh[1] = prv.y;
  wl[0] = prv.z;
  wl[1] = prv.w;
  wh[L + 2] = nxt.x;
  wh[L + 3] = nxt.y;
  wl[L + 2] = nxt.z;
  wl[L + 3] = nxt.w;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    wh[j + 2] = ch[j];
    wl[j + 2] = cl[j];
  }
  if (PER) {
    fill_wrap<L>(wh, wl, tg, n, wrap_slots(cx, sm));
  } else {
    fill_ghosts<L>(wh, tg, n);
    fill_ghosts<L>(wl, tg, n);
  }
  float uh[L + 2], ul[L + 2];  // C^3 - C at rows tg L - 1 .. tg L + L
  if (has_mu) {
#pragma unroll
    for (int q = 0; q < L + 2; ++q) cube_minus_ff(wh[q + 1], wl[q + 1], uh[q], ul[q]);
  }
#pragma unroll
  for (int j = 0; j < L; ++j) {
    float sh = twice ? 2.f * wh[j + 2] : wh[j + 2], sl = twice ? 2.f * wl[j + 2] : wl[j + 2];
    if (has_mu) {
      float dh, dl, ph, pl, a, e;
      d2_ff(uh[j], ul[j], uh[j + 2], ul[j + 2], uh[j + 1], ul[j + 1], dh, dl);
      mul_ff(muh, mul, dh, dl, ph, pl);
      two_sum(sh, ph, a, e);
      fast_two_sum(a, e + (sl + pl), sh, sl);
    }
    if (has_nu && !twice) {
      float yh, yl, ph, pl, a, e;
      d4_ff(wh[j], wl[j], wh[j + 1], wl[j + 1], wh[j + 2], wl[j + 2], wh[j + 3], wl[j + 3], wh[j + 4], wl[j + 4], yh,
            yl);
      mul_ff(nuh, nul, yh, yl, ph, pl);
      two_sum(sh, -ph, a, e);
      fast_two_sum(a, e + (sl - pl), sh, sl);
    }
    const bool in = tg * L + j < n;
    fh[j] = in ? sh : 0.f;
    fl[j] = in ? sl : 0.f;
  }
}

// Load the thread's 1/alpha and beta (stored as float4 planes, see k_factor32).
// gq: the system's factor block; PT threads per system; tg this thread's index.
// NPL: float4 planes per group of four rows (2; periodic systems 4: their
// blocks also hold the two columns of Z, see k_factor32_periodic).
template <int L, int NPL = 2>
__device__ __forceinline__ void load_factors(Fac<L>& fc, const float4* __restrict__ gq, int tg, int PT) {
#pragma unroll
  for (int jq = 0; jq < L / 4; ++jq) {
    const float4 qa = __ldg(gq + (int64_t)(jq * NPL + 0) * PT + tg),
                 qb = __ldg(gq + (int64_t)(jq * NPL + 1) * PT + tg);
    fc.A[4 * jq] = qa.x; fc.A[4 * jq + 1] = qa.y; fc.A[4 * jq + 2] = qa.z; fc.A[4 * jq + 3] = qa.w;
    fc.Bt[4 * jq] = qb.x; fc.Bt[4 * jq + 1] = qb.y; fc.Bt[4 * jq + 2] = qb.z; fc.Bt[4 * jq + 3] = qb.w;
  }
  fc.bnext = (tg + 1 < PT) ? __ldg(reinterpret_cast<const float*>(gq + (int64_t)PT + (tg + 1))) : 0.f;
}

// One CTA (or one cluster of C CTAs) per system: FP32 solve, then up to
// max_refine refinement steps.  RES64 selects the FP64 residual (and FP64
// accumulation of x) instead of float-float.
// Refinement stops early once the error left after a step, estimated as the
// step's correction times the contraction of the iteration, is below
// 2^-tol_log2 max|x|; the contraction is estimated by max|dx| / max|x| and, from
// the second step on, by the ratio of successive corrections if that is larger.
// WT > 0 fixes the warp count at compile time (the common one-CTA shapes);
// WT = 0 takes it from `Wrt`.  CL enables the cluster paths (C = Crt CTAs per
// system), otherwise C = 1.  Register budget: 6 CTAs of 4 warps per SM (at most
// 85 registers a thread; the few that spill cost less than the latency the
// extra CTA hides: 0.63 against 0.70 ms per parametric step at 5 CTAs).
constexpr int min_blocks(int L, int WT, bool STEP) {
  return WT > 0 ? ((L <= 8 && (STEP ? 20 : 24) / WT > 0) ? (STEP ? 20 : 24) / WT : 1) : 1;
}

// STEP: the right-hand side is not given but assembled from the field in f as
// f = C + mu_s D2(C^3 - C) - nu_s D4 C (step_rhs_ff), with no scaling (the field
// must stay below 2^40 in magnitude; larger values are flagged as not converged);
// x (normally = f) receives the new field.
// PER: a periodic system (Sec. 2.3): the factors are those of the leading
// n - 2 rows E with two more planes holding Z = E^{-1} k, each FP32 solve is
// followed by Navon's tail (periodic_tail), and the residual and the
// right-hand side take wrapped neighbours.
template <int L, int WT, bool CL, bool RES64, bool STEP = false, bool PER = false>
__global__ void __launch_bounds__(WT > 0 ? 32 * WT : 512, min_blocks(L, WT, STEP || PER))
    k_solve32r(F32Tables T, const int32_t* __restrict__ sys, int Wrt, int Crt, int shared, const double* f, double* x,
               int max_refine, int tol_log2, int vec_io, const double* __restrict__ mu_s,
               const double* __restrict__ nu_s) {
  static_assert(L % 4 == 0, "rows per thread must be a multiple of 4");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = WT > 0 ? WT : Wrt;
  const int C = CL ? Crt : 1;
  const SmemView sm = smem_view(smem_raw, W);
  const int P = 32 * W, PT = P * C;
  const int t = threadIdx.x;
  Ctx cx;
  cx.lane = t & 31;
  cx.warp = t >> 5;
  cx.t = t;
  cx.P = P;
  cx.W = W;
  cx.C = C;
  cx.rank = (C > 1) ? (int)cg::this_cluster().block_rank() : 0;
  cx.phase = 0;
  const int64_t s = sys[blockIdx.x / C];
  const int64_t ms = shared ? 0 : s;
  const int n = T.n[s];
  const int tg = cx.rank * P + t;

  // ---- loads: factors, right-hand side (all coalesced) ----
  const float2 sgp = __ldg(T.sig2 + ms);  // sigma as an FP32 pair, split at factorisation time
  const float sgh = sgp.x, sgl = sgp.y;
  Fac<L> fc;
  fc.sg = sgh;
  constexpr int NPL = PER ? 4 : 2;
  const float4* __restrict__ gq = reinterpret_cast<const float4*>(T.fac) + T.foff[ms];
  load_factors<L, NPL>(fc, gq, tg, PT);
  const float4 psi = PER ? __ldg(T.psinv + ms) : make_float4(0.f, 0.f, 0.f, 0.f);
  const double* fs = f + T.off[s];
  const int i0 = tg * L;
  double fv[L];
  if (vec_io && i0 + L <= n) {
#pragma unroll
    for (int j = 0; j < L; j += 2) {
      const double2 q = *reinterpret_cast<const double2*>(fs + i0 + j);
      fv[j] = q.x;
      fv[j + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j) fv[j] = (i0 + j < n) ? fs[i0 + j] : 0.0;
  }

  // ---- scan plan of both sweeps (factors only) ----
  cx.nlev[0] = scan_setup<true>(fwd_chunk_map<L>(fc), cx, sm);
  cx.nlev[1] = scan_setup<false>(bwd_chunk_map<L>(fc), cx, sm);

  // ---- per-system power-of-two scale: the largest |f| maps just below 1 ----
  int emax = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const unsigned top = (unsigned)((unsigned long long)__double_as_longlong(fv[j]) >> 32);
    emax = max(emax, (int)((top >> 20) & 0x7ffu));
  }
  // (the barrier inside also orders the scan plan's writes before any read)
  emax = system_max<int>(emax, cx.lane, cx.warp, W, C, sm.redi);
  if (C > 1 && t == 0) cta_total_maps(cx, sm);  // read by the other CTAs after the first scan's cluster barrier
  const int kshift = STEP ? 0 : emax - 1022;

  float v[L], xh[L], xl[L];
  float fh[L], fl[L];
  // Crank-Nicolson with nu = sigma: solve for 2 C + mu D2(C^3 - C), subtract C at the end
  const bool twice = STEP && nu_s && nu_s[ms] == T.sigma[ms];
  if (STEP) {
    float muh = 0.f, mul = 0.f, nuh = 0.f, nul = 0.f;
    if (mu_s) split_scaled(mu_s[ms], 0, muh, mul);
    if (nu_s) split_scaled(nu_s[ms], 0, nuh, nul);
    if (emax >= 1023 + 40 && t == 0) atomicOr(T.info + 2, 1ull);  // |C| >= 2^40: outside the FP32 path's range
    step_rhs_ff<L, PER>(fv, muh, mul, nuh, nul, muh != 0.f, nuh != 0.f, twice, fh, fl, n, tg, cx, sm);
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j) split_scaled(fv[j], kshift, fh[j], fl[j]);
  }
#pragma unroll
  for (int j = 0; j < L; ++j) v[j] = fh[j];
  int steps = 0;
  bool stalled = false;
  const float tol = ldexpf(1.0f, -tol_log2);
  float prev = INFINITY;
  if (RES64) {
    // x kept in FP64 (scaled by 2^-kshift); f in FP64 scaled the same way
    double xd[L], fd[L];
    const double scale = ldexp(1.0, -kshift);
    const double sg = T.sigma[ms];
#pragma unroll
    for (int j = 0; j < L; ++j) fd[j] = fv[j] * scale;
#pragma unroll 1
    for (int it = 0; it <= max_refine; ++it) {
      if (it > 0) residual_f64<L>(fd, xd, v, sg, n, tg, cx, sm);
      cta_solve32<L>(v, fc, cx, sm);
      if (it == 0) {
#pragma unroll
        for (int j = 0; j < L; ++j) xd[j] = (double)v[j];
        continue;
      }
      float dmax = 0.f, xmax = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        xd[j] += (double)v[j];
        dmax = fmaxf(dmax, fabsf(v[j]));
        xmax = fmaxf(xmax, fabsf((float)xd[j]));
      }
      steps = it;
      if (it < max_refine) {
        float* rs = sm.red + (cx.phase++ & 3) * (W + 1);
        dmax = system_max<float>(dmax, cx.lane, cx.warp, W, C, rs);
        float* rs2 = sm.red + (cx.phase++ & 3) * (W + 1);
        xmax = system_max<float>(xmax, cx.lane, cx.warp, W, C, rs2);
        // error left ~ dmax times the contraction per step, estimated by the correction's size
        // relative to x and, from the second step on, by the ratio of successive corrections
        // (the larger: at large condition numbers the first underestimates it)
        const float q = dmax / xmax;
        const float rho = (it > 1 && prev > 0.f) ? fmaxf(q, dmax / prev) : q;
        if (!(dmax > 0.f) || dmax * rho <= tol * xmax) break;
        if (it > 1 && dmax > 0.5f * prev) {
          stalled = true;
          break;
        }
        prev = dmax;
      }
    }
#pragma unroll
    for (int j = 0; j < L; ++j) fv[j] = ldexp(xd[j], kshift);
  } else {
    // it = 0 solves for f (its FP32 part); every later pass solves for the
    // float-float residual of the current x and adds the correction.  One
    // solve call site keeps the unrolled kernel compact (instruction cache).
#pragma unroll 1
    for (int it = 0; it <= max_refine; ++it) {
      if (PER) {
        if (it == 1)
          residual_ff_per<L, true>(fh, fl, xh, xl, v, sgh, sgl, n, tg, cx, sm);
        else if (it > 1)
          residual_ff_per<L, false>(fh, fl, xh, xl, v, sgh, sgl, n, tg, cx, sm);
        periodic_tail_rhs<L>(v, tg, n, cx, sm);
        cta_solve32<L>(v, fc, cx, sm);
        periodic_tail<L, NPL>(v, gq, PT, tg, n, sgh, psi, cx, sm);
      } else {
        if (it == 1)
          residual_ff<L, true>(fh, fl, xh, xl, v, sgh, sgl, n, tg, cx, sm);  // x is still one float per row
        else if (it > 1)
          residual_ff<L, false>(fh, fl, xh, xl, v, sgh, sgl, n, tg, cx, sm);
        cta_solve32<L>(v, fc, cx, sm);
      }
      if (it == 0) {
#pragma unroll
        for (int j = 0; j < L; ++j) {
          xh[j] = v[j];
          xl[j] = 0.f;
        }
        continue;
      }
      float dmax = 0.f, xmax = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        float sh, se;
        two_sum(xh[j], v[j], sh, se);
        se = se + xl[j];
        fast_two_sum(sh, se, xh[j], xl[j]);
        dmax = fmaxf(dmax, fabsf(v[j]));
        xmax = fmaxf(xmax, fabsf(xh[j]));
      }
      steps = it;
      if (it < max_refine) {  // the stopping tests only matter if another step may follow
        float* rs = sm.red + (cx.phase++ & 3) * (W + 1);
        dmax = system_max<float>(dmax, cx.lane, cx.warp, W, C, rs);
        float* rs2 = sm.red + (cx.phase++ & 3) * (W + 1);
        xmax = system_max<float>(xmax, cx.lane, cx.warp, W, C, rs2);
        // error left ~ dmax times the contraction per step, estimated by the correction's size
        // relative to x and, from the second step on, by the ratio of successive corrections
        // (the larger: at large condition numbers the first underestimates it)
        const float q = dmax / xmax;
        const float rho = (it > 1 && prev > 0.f) ? fmaxf(q, dmax / prev) : q;
        if (!(dmax > 0.f) || dmax * rho <= tol * xmax) break;
        if (it > 1 && dmax > 0.5f * prev) {
          stalled = true;
          break;
        }
        prev = dmax;
      }
    }
    if (twice) {  // C' = A^{-1}(2 C + ...) - C, in float-float; C is re-read (this thread's rows are unchanged)
#pragma unroll
      for (int j = 0; j < L; ++j) {
        float ch, cl, sh, se;
        split_scaled((i0 + j < n) ? fs[i0 + j] : 0.0, 0, ch, cl);
        two_sum(xh[j], -ch, sh, se);
        fast_two_sum(sh, se + (xl[j] - cl), xh[j], xl[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < L; ++j) fv[j] = ff_to_double_shift(xh[j], xl[j], kshift);
  }
  if (t == 0 && cx.rank == 0) {
    if (steps > 0) atomicMax(T.info + 1, (unsigned long long)steps);
    if (stalled) atomicOr(T.info + 2, 1ull);
  }
  // ---- store x (a thread's rows are contiguous) ----
  double* xs = x + T.off[s];
  if (vec_io && i0 + L <= n) {
#pragma unroll
    for (int j = 0; j < L; j += 2) *reinterpret_cast<double2*>(xs + i0 + j) = make_double2(fv[j], fv[j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j)
      if (i0 + j < n) xs[i0 + j] = fv[j];
  }
  if (C > 1) cg::this_cluster().sync();  // keep this CTA's shared memory alive for the cluster's readers
}

// Factor A = I + sigma D4 of one system per thread in FP64 (Sec. 2.4,
// factorisation steps 1-14) and store 1/alpha and beta rounded to FP32 in the
// system's block: float4 ((j / 4) * 2 + p) * PT + tg holds rows tg L + 4 (j/4)
// .. + 3 of plane p (0: 1/alpha, 1: beta), PT threads of L rows per system.
__global__ void k_factor32(F32Tables T, int64_t nsys, const int32_t* __restrict__ shape,
                           const double* __restrict__ sigma) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const int n = T.n[s];
  const int PT = shape[s] & 0xffff, L = shape[s] >> 16;
  const double sg = sigma[s];
  {
    const float hi = __double2float_rn(sg);
    T.sig2[s] = make_float2(hi, __double2float_rn(sg - (double)hi));
  }
  float* F = T.fac + T.foff[s] * 4;
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;
  bool failed = false;
  const int rows = PT * L;
  for (int i = 0; i < rows; ++i) {
    float ainv = 0.f, bt = 0.f;  // padding rows and rows after a failed pivot: g = x = 0
    if (i < n && !failed) {
      double ar = sg, br = -4.0 * sg, cr = 1.0 + sg * 6.0, dr = -4.0 * sg, er = sg;  // interior rows
      if (i < 2 || i + 2 >= n) {  // the two rows at each wall
        float w[5];
        d4_weights_f(i, n, w);
        ar = (i >= 2) ? sg * w[0] : 0.0;
        br = (i >= 1) ? sg * w[1] : 0.0;
        cr = 1.0 + sg * w[2];
        dr = (i + 1 < n) ? sg * w[3] : 0.0;
        er = (i + 2 < n) ? sg * w[4] : 0.0;
      }
      const double beta = br - ar * gam2;
      const double alpha = cr - ar * del2 - beta * gam1;
      if (!(alpha != 0.0) || !isfinite(alpha)) {
        const unsigned long long key = ((unsigned long long)s << 32) | (unsigned long long)(uint32_t)i;
        atomicMin(T.info, key);
        failed = true;
      } else {
        const double gamma = (dr - beta * del1) / alpha;
        const double delta = er / alpha;
        ainv = (float)(1.0 / alpha);
        bt = (float)beta;
        gam2 = gam1;
        del2 = del1;
        gam1 = gamma;
        del1 = delta;
      }
    }
    const int tgi = i / L, j = i - tgi * L;
    const int64_t base = ((int64_t)(j / 4) * 2) * PT * 4 + (int64_t)tgi * 4 + (j & 3);
    F[base] = ainv;
    F[base + (int64_t)PT * 4] = bt;
  }
}

// Factor the periodic matrix of Eq. (matrix_sys) for FP32 solves, one thread per
// system (FP64 arithmetic): E, its first m = n - 2 rows and columns (the band
// cut off at E's edges), by the Sec. 2.4 steps, stored as 1/alpha and beta in
// planes 0, 1 of a 4-plane block (float4 ((j / 4) * 4 + p) * PT + tg); rows m and
// m + 1 and padding rows are zero.  Planes 2, 3: the columns of
// Z = E^{-1} k, computed as W = L^{-1} k (forward, FP64) then R Z = W (back, with
// the stored FP32 factors, as the solve uses them); k's nonzeros are a_0 = sigma,
// e_{m-2} = sigma, d_{m-1} = -4 sigma (column n-2) and b_0 = -4 sigma,
// a_1 = sigma, e_{m-1} = sigma (column n-1).  S^{-1} = (D - h^T Z)^{-1} (h = k,
// the matrix being symmetric) goes to psinv.
__global__ void k_factor32_periodic(F32Tables T, int64_t nsys, const int32_t* __restrict__ shape,
                                    const double* __restrict__ sigma) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const int n = T.n[s], m = n - 2;
  const int PT = shape[s] & 0xffff, L = shape[s] >> 16;
  const double sg = sigma[s];
  {
    const float hi = __double2float_rn(sg);
    T.sig2[s] = make_float2(hi, __double2float_rn(sg - (double)hi));
  }
  float* F = T.fac + T.foff[s] * 4;
  auto at = [&](int i, int p) -> float& {
    const int tgi = i / L, j = i - tgi * L;
    return F[((int64_t)(j / 4) * 4 + p) * PT * 4 + (int64_t)tgi * 4 + (j & 3)];
  };
  const int rows = PT * L;
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;
  double w02 = 0.0, w01 = 0.0, w12 = 0.0, w11 = 0.0;  // W of rows i-2, i-1 (both columns)
  bool failed = false;
  for (int i = 0; i < rows; ++i) {
    float ainv = 0.f, bt = 0.f, wa = 0.f, wb = 0.f;
    if (i < m && !failed) {
      const double ar = (i >= 2) ? sg : 0.0, br = (i >= 1) ? -4.0 * sg : 0.0, cr = 1.0 + 6.0 * sg;
      const double dr = (i + 1 < m) ? -4.0 * sg : 0.0, er = (i + 2 < m) ? sg : 0.0;
      const double beta = br - ar * gam2;
      const double alpha = cr - ar * del2 - beta * gam1;
      if (!(alpha != 0.0) || !isfinite(alpha)) {
        atomicMin(T.info, ((unsigned long long)s << 32) | (unsigned long long)(uint32_t)i);
        failed = true;
      } else {
        const double k0 = (i == 0 ? sg : 0.0) + (i == m - 2 ? sg : 0.0) + (i == m - 1 ? -4.0 * sg : 0.0);
        const double k1 = (i == 0 ? -4.0 * sg : 0.0) + (i == 1 ? sg : 0.0) + (i == m - 1 ? sg : 0.0);
        const double w0 = (k0 - ar * w02 - beta * w01) / alpha;
        const double w1 = (k1 - ar * w12 - beta * w11) / alpha;
        w02 = w01;
        w01 = w0;
        w12 = w11;
        w11 = w1;
        const double gamma = (dr - beta * del1) / alpha;
        const double delta = er / alpha;
        ainv = (float)(1.0 / alpha);
        bt = (float)beta;
        wa = (float)w0;
        wb = (float)w1;
        gam2 = gam1;
        del2 = del1;
        gam1 = gamma;
        del1 = delta;
      }
    }
    at(i, 0) = ainv;
    at(i, 1) = bt;
    at(i, 2) = wa;
    at(i, 3) = wb;
  }
  // R Z = W: z_i = w_i - gamma_i z_{i+1} - delta_i z_{i+2}, gamma_i = beta_{i+1} / alpha_i,
  // delta_i = sigma / alpha_i (zero past E's edge, where z is zero anyway)
  double z01 = 0.0, z02 = 0.0, z11 = 0.0, z12 = 0.0;  // z of rows i+1, i+2
  for (int i = m - 1; i >= 0; --i) {
    const double ia = (double)at(i, 0);
    const double gamma = (i + 1 < m) ? (double)at(i + 1, 1) * ia : 0.0;
    const double delta = sg * ia;
    const double z0 = (double)at(i, 2) - gamma * z01 - delta * z02;
    const double z1 = (double)at(i, 3) - gamma * z11 - delta * z12;
    at(i, 2) = (float)z0;
    at(i, 3) = (float)z1;
    z02 = z01;
    z01 = z0;
    z12 = z11;
    z11 = z1;
  }
  // S = D - h^T Z, h^T's rows: (sigma @ 0, sigma @ m-2, -4 sigma @ m-1), (-4 sigma @ 0, sigma @ 1, sigma @ m-1)
  auto hz = [&](int c, int row) {
    const double za = at(0, 2 + c), zb = at(1, 2 + c), zm2 = at(m - 2, 2 + c), zm1 = at(m - 1, 2 + c);
    return row == 0 ? sg * (za + zm2) - 4.0 * sg * zm1 : -4.0 * sg * za + sg * (zb + zm1);
  };
  const double s00 = 1.0 + 6.0 * sg - hz(0, 0), s01 = -4.0 * sg - hz(1, 0);
  const double s10 = -4.0 * sg - hz(0, 1), s11 = 1.0 + 6.0 * sg - hz(1, 1);
  const double det = s00 * s11 - s01 * s10;
  if (failed || !(det != 0.0) || !isfinite(det)) {
    if (!failed) atomicMin(T.info, ((unsigned long long)s << 32) | (unsigned long long)(uint32_t)(n - 2));
    T.psinv[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  T.psinv[s] = make_float4((float)(s11 / det), (float)(-s01 / det), (float)(-s10 / det), (float)(s00 / det));
}

template <int L, int WT, bool CL, bool RES64, bool STEP, bool PER = false>
cudaError_t launch_bucket(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                          double* x, int max_refine, int tol_log2, const double* mu, const double* nu,
                          cudaStream_t st) {
  const int vec = ((((uintptr_t)f) | ((uintptr_t)x)) % 16 == 0) && b.even_offsets;
  const size_t smem = smem_bytes(b.W);
  if (smem > 48 * 1024) {  // above the default dynamic shared memory limit (a function attribute, not a stream op)
    const cudaError_t e = cudaFuncSetAttribute(k_solve32r<L, WT, CL, RES64, STEP, PER>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b.count * b.C));
  cfg.blockDim = dim3(32 * b.W);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (b.C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = b.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, k_solve32r<L, WT, CL, RES64, STEP, PER>, T, sys + b.first, b.W, b.C, shared, f, x,
                            max_refine, tol_log2, vec, mu, nu);
}

template <int L, bool RES64, bool STEP>
cudaError_t dispatch_bucket(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                            double* x, int max_refine, int tol_log2, const double* mu, const double* nu,
                            cudaStream_t st) {
  if (b.C > 1) {
    // clusters of 4- or 8-warp CTAs compiled for that width (several CTAs per SM), else any width
    if (!RES64 && b.W == 4)
      return launch_bucket<L, 4, true, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
    if (!RES64 && b.W == 8)
      return launch_bucket<L, 8, true, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
    return launch_bucket<L, 0, true, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
  }
  if (!RES64) {
    switch (b.W) {
      case 1: return launch_bucket<L, 1, false, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
      case 2: return launch_bucket<L, 2, false, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
      case 4: return launch_bucket<L, 4, false, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
      case 8: return launch_bucket<L, 8, false, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
      case 16:
        return launch_bucket<L, 16, false, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
      default: break;
    }
  }
  return launch_bucket<L, 0, false, RES64, STEP>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
}

}  // namespace

cudaError_t launch_factor32(const F32Tables& T, const int32_t* shape, int64_t nsys, const double* sigma,
                            cudaStream_t st) {
  const int block = 128;
  k_factor32<<<(unsigned)((nsys + block - 1) / block), block, 0, st>>>(T, nsys, shape, sigma);
  return cudaGetLastError();
}

// Periodic systems: one kernel shape for every CTA width (the runtime-W form), clusters when needed.
template <int L, bool STEP>
cudaError_t dispatch_periodic(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                              double* x, int max_refine, int tol_log2, const double* mu, const double* nu,
                              cudaStream_t st) {
  if (b.C > 1)
    return launch_bucket<L, 0, true, false, STEP, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
  if (b.W == 2)
    return launch_bucket<L, 2, false, false, STEP, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
  if (b.W == 4)
    return launch_bucket<L, 4, false, false, STEP, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
  return launch_bucket<L, 0, false, false, STEP, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
}

cudaError_t launch_solve32r(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                            double* x, int max_refine, int residual_f64, int tol_log2, cudaStream_t st,
                            const double* mu, const double* nu, bool step, bool periodic) {
  if (b.count == 0) return cudaSuccess;
  if (periodic) {  // float-float residual only
    if (residual_f64) return cudaErrorInvalidValue;
    if (b.L == 4)
      return step ? dispatch_periodic<4, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st)
                  : dispatch_periodic<4, false>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
    if (b.L == 8)
      return step ? dispatch_periodic<8, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st)
                  : dispatch_periodic<8, false>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
    return cudaErrorInvalidValue;
  }
  if (step) {  // float-float residual only
    if (residual_f64) return cudaErrorInvalidValue;
    if (b.L == 4) return dispatch_bucket<4, false, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
    if (b.L == 8) return dispatch_bucket<8, false, true>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
    return cudaErrorInvalidValue;
  }
  if (b.L == 4)
    return residual_f64 ? dispatch_bucket<4, true, false>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st)
                        : dispatch_bucket<4, false, false>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
  if (b.L == 8)
    return residual_f64 ? dispatch_bucket<8, true, false>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st)
                        : dispatch_bucket<8, false, false>(T, sys, b, shared, f, x, max_refine, tol_log2, mu, nu, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_factor32_periodic(const F32Tables& T, const int32_t* shape, int64_t nsys, const double* sigma,
                                     cudaStream_t st) {
  const int block = 128;
  k_factor32_periodic<<<(unsigned)((nsys + block - 1) / block), block, 0, st>>>(T, nsys, shape, sigma);
  return cudaGetLastError();
}

}  // namespace pent
