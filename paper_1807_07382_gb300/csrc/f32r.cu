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
// One CTA of P = 32 W threads owns one system of n <= P L rows: thread t holds
// rows t L .. t L + L - 1, their factors and their right-hand side in registers
// (all loaded with coalesced 16-byte accesses, since a thread's rows are
// contiguous).  Each substitution (Sec. 2.4: L g = f, then R x = g) is a
// second-order linear recurrence, so a thread's chunk acts on the two carried
// values as an affine map.  The thread runs its chunk from a zero state to get
// the affine part; the CTA composes the maps with a Kogge-Stone shuffle scan in
// each warp and a short carry across warps; then every thread reruns its chunk
// from the true entering state.  The factors are read from HBM once per call
// and reused by every substitution of every refinement step.
//
// The hyperdiffusion matrices are symmetric, so A = L D^{-1} L^T with D the
// diagonal alpha of L: R = D^{-1} L^T, gamma_i = beta_{i+1} / alpha_i and
// delta_i = epsilon_{i+2} / alpha_i, and epsilon_i = a_i is sigma times a
// stencil weight.  Only 1/alpha_i and beta_i are stored (8 bytes per row in
// FP32); epsilon, gamma, delta and the chunks' 2x2 transfer maps are rebuilt in
// registers, trading FP32 arithmetic for HBM bytes.
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace pent {
namespace {

// ---------------------------------------------------------------- error-free transformations (FP32)

// s + e == a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e == a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// p + e == a * b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// float from a small non-negative integer (< 2^23) without a conversion instruction.
__device__ __forceinline__ float small_uint_to_float(unsigned v) {
  return __fsub_rn(__uint_as_float(0x4b000000u | v), 8388608.0f);
}

// v * 2^-k split into hi + lo floats (hi: v truncated to 24 significant bits,
// lo: the next 24 bits, rounded), using integer operations only.  Values whose
// scaled magnitude is below 2^-126 are flushed to zero; the caller picks k so
// that the largest |v| of the system scales to just below 1.
__device__ __forceinline__ void split_scaled(double v, int k, float& hi, float& lo) {
  const unsigned long long U = (unsigned long long)__double_as_longlong(v);
  const unsigned top = (unsigned)(U >> 32);
  const int E = (int)((top >> 20) & 0x7ffu);
  const int Es = E - k;
  const unsigned sign = top & 0x80000000u;
  if (E == 0 || Es < 897) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  const unsigned mant_hi = (unsigned)((U >> 29) & 0x7fffffu);
  hi = __uint_as_float(sign | ((unsigned)(Es - 896) << 23) | mant_hi);
  if (Es < 949) {
    lo = 0.0f;
    return;
  }
  const unsigned rem = (unsigned)(U & 0x1fffffffu);  // low 29 mantissa bits
  const float r = __fmaf_rn(small_uint_to_float(rem >> 6), 64.0f, small_uint_to_float(rem & 63u));
  const float scale = __uint_as_float((unsigned)(Es - 948) << 23);  // 2^(Es - 1075)
  lo = __uint_as_float(__float_as_uint(__fmul_rn(r, scale)) ^ sign);
}

// Rare path of f2d_shift (subnormal float or a result outside the normal double
// range).  Kept out of line so that its FP64 arithmetic is never if-converted
// into the common path.
__device__ __noinline__ double f2d_shift_slow(float v, int k) { return ldexp((double)v, k); }

// Exact v * 2^k as a double, by moving v's exponent and mantissa bit fields.
__device__ __forceinline__ double f2d_shift(float v, int k) {
  const unsigned u = __float_as_uint(v);
  const unsigned a = u & 0x7fffffffu;
  if (a == 0u) return 0.0;
  const int e = (int)(a >> 23);
  const int de = e + 896 + k;
  if (e == 0 || e == 255 || de < 1 || de > 2046) return f2d_shift_slow(v, k);
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  (((unsigned long long)a + ((unsigned long long)(896 + k) << 23)) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

// Weights of the no-flux fourth difference on row i (n rows), reflected about
// the cell-centred walls; w[k] multiplies x_{i+k-2}.  Small integers.
__device__ __forceinline__ void d4_weights_f(int i, int n, float w[5]) {
  const float st[5] = {1.f, -4.f, 6.f, -4.f, 1.f};
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    int j = i + k - 2;
    while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
    w[j - i + 2] += st[k];
  }
}

// ---------------------------------------------------------------- CTA-wide affine scans

// x -> [[a, b], [c, d]] x + (u, v): the effect of a chunk of rows on the two carried values.
struct Aff {
  float a, b, c, d, u, v;
};

// `later` applied after `earlier`.
__device__ __forceinline__ Aff compose(const Aff& L, const Aff& E) {
  Aff r;
  r.a = fmaf(L.a, E.a, L.b * E.c);
  r.b = fmaf(L.a, E.b, L.b * E.d);
  r.c = fmaf(L.c, E.a, L.d * E.c);
  r.d = fmaf(L.c, E.b, L.d * E.d);
  r.u = fmaf(L.a, E.u, fmaf(L.b, E.v, L.u));
  r.v = fmaf(L.c, E.u, fmaf(L.d, E.v, L.v));
  return r;
}

template <bool UP>
__device__ __forceinline__ Aff shfl_aff(const Aff& x, int d) {
  Aff r;
  if (UP) {
    r.a = __shfl_up_sync(0xffffffffu, x.a, d);
    r.b = __shfl_up_sync(0xffffffffu, x.b, d);
    r.c = __shfl_up_sync(0xffffffffu, x.c, d);
    r.d = __shfl_up_sync(0xffffffffu, x.d, d);
    r.u = __shfl_up_sync(0xffffffffu, x.u, d);
    r.v = __shfl_up_sync(0xffffffffu, x.v, d);
  } else {
    r.a = __shfl_down_sync(0xffffffffu, x.a, d);
    r.b = __shfl_down_sync(0xffffffffu, x.b, d);
    r.c = __shfl_down_sync(0xffffffffu, x.c, d);
    r.d = __shfl_down_sync(0xffffffffu, x.d, d);
    r.u = __shfl_down_sync(0xffffffffu, x.u, d);
    r.v = __shfl_down_sync(0xffffffffu, x.v, d);
  }
  return r;
}

// Coupling below this norm is dropped from the scans: it changes the carried
// values by less than FP32 resolution, and the refinement corrects the FP32
// solve anyway.
constexpr float kScanTol = 9.3132257e-10f;  // 2^-30

__device__ __forceinline__ float mat_norm(const Aff& m) {
  return fmaxf(fmaxf(fabsf(m.a), fabsf(m.b)), fmaxf(fabsf(m.c), fabsf(m.d)));
}

// Entering state of this thread's chunk for a sweep through the CTA's chunks.
// FWD: chunks are visited in increasing thread order; otherwise decreasing.
// `a` is this chunk's map (linear part from the factors, affine part from a
// zero-state pass).  The system is entered with state 0.  The Kogge-Stone
// levels stop as soon as every lane's window either reaches the warp's first
// chunk or composes to a negligible linear part, since later levels would only
// add terms multiplied by it.  sh: 2 float4 per warp.
template <int W, bool FWD>
__device__ __forceinline__ void scan_entry(Aff a, int lane, int warp, float4* sh, float& e0, float& e1) {
#pragma unroll 1
  for (int d = 1; d < 32; d <<= 1) {
    const Aff o = shfl_aff<FWD>(a, d);
    if (FWD ? (lane >= d) : (lane + d < 32)) a = compose(a, o);
    const bool done = (FWD ? (lane < 2 * d) : (lane + 2 * d > 31)) || mat_norm(a) < kScanTol;
    if (__all_sync(0xffffffffu, done)) break;
  }
  const Aff prev = shfl_aff<FWD>(a, 1);  // inclusive result of the previous chunk in sweep order
  const bool first = FWD ? (lane == 0) : (lane == 31);
  float c0 = 0.f, c1 = 0.f;  // state entering this warp
  if (W > 1) {
    if (FWD ? (lane == 31) : (lane == 0)) {
      sh[2 * warp] = make_float4(a.a, a.b, a.c, a.d);
      sh[2 * warp + 1] = make_float4(a.u, a.v, 0.f, 0.f);
    }
    __syncthreads();
    if (FWD) {
      for (int w = 0; w < warp; ++w) {
        const float4 m = sh[2 * w], b = sh[2 * w + 1];
        const float n0 = fmaf(m.x, c0, fmaf(m.y, c1, b.x));
        const float n1 = fmaf(m.z, c0, fmaf(m.w, c1, b.y));
        c0 = n0;
        c1 = n1;
      }
    } else {
      for (int w = W - 1; w > warp; --w) {
        const float4 m = sh[2 * w], b = sh[2 * w + 1];
        const float n0 = fmaf(m.x, c0, fmaf(m.y, c1, b.x));
        const float n1 = fmaf(m.z, c0, fmaf(m.w, c1, b.y));
        c0 = n0;
        c1 = n1;
      }
    }
  }
  if (first) {
    e0 = c0;
    e1 = c1;
  } else {
    e0 = fmaf(prev.a, c0, fmaf(prev.b, c1, prev.u));
    e1 = fmaf(prev.c, c0, fmaf(prev.d, c1, prev.v));
  }
}

template <int W>
__device__ __forceinline__ float block_max(float v, int lane, int warp, float* sh) {
  v = warp_max(v);
  if (W == 1) return v;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float r = sh[0];
#pragma unroll
  for (int w = 1; w < W; ++w) r = fmaxf(r, sh[w]);
  return r;
}

template <int W>
__device__ __forceinline__ int block_max_i(int v, int lane, int warp, int* sh) {
  v = warp_max_i(v);
  if (W == 1) return v;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  int r = sh[0];
#pragma unroll
  for (int w = 1; w < W; ++w) r = max(r, sh[w]);
  return r;
}

// Shared scratch of one CTA.  Scan and reduction slots rotate through four
// buffers, so a single barrier per scan separates every write from the reads
// of the same buffer.
template <int W>
struct Smem {
  float4 scan[4][2 * W];
  float4 edge[32 * W][2];  // per thread: first two rows (hi, lo), last two rows (hi, lo)
  float red[4][2 * W];
  int redi[W];
};

// Per-thread factors of its L rows and the chunk maps, rebuilt from the stored
// 1/alpha and beta (see the header comment).
template <int L>
struct ChunkFactors {
  float A[L];  // 1/alpha_i
  float B[L];  // beta_i / alpha_i
  float E[L];  // epsilon_i / alpha_i
  float G[L];  // gamma_i
  float D[L];  // delta_i
  float4 pf;   // forward map (row-major 2x2)
  float4 pb;   // backward map
};

// In place v <- A^{-1} v (FP32): forward L g = v, then back R x = g.
template <int W, int L>
__device__ __forceinline__ void cta_solve32(float (&v)[L], const ChunkFactors<L>& cf, int lane, int warp, Smem<W>& sm,
                                            int& phase) {
  float p2 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float g = fmaf(-cf.B[j], p1, fmaf(-cf.E[j], p2, cf.A[j] * v[j]));
    p2 = p1;
    p1 = g;
  }
  float e0, e1;
  scan_entry<W, true>(Aff{cf.pf.x, cf.pf.y, cf.pf.z, cf.pf.w, p2, p1}, lane, warp, sm.scan[phase++ & 3], e0, e1);
  p2 = e0;
  p1 = e1;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float g = fmaf(-cf.B[j], p1, fmaf(-cf.E[j], p2, cf.A[j] * v[j]));
    v[j] = g;
    p2 = p1;
    p1 = g;
  }
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const float xv = fmaf(-cf.G[j], s1, fmaf(-cf.D[j], s2, v[j]));
    s2 = s1;
    s1 = xv;
  }
  scan_entry<W, false>(Aff{cf.pb.x, cf.pb.y, cf.pb.z, cf.pb.w, s1, s2}, lane, warp, sm.scan[phase++ & 3], e0, e1);
  s1 = e0;
  s2 = e1;
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const float xv = fmaf(-cf.G[j], s1, fmaf(-cf.D[j], s2, v[j]));
    v[j] = xv;
    s2 = s1;
    s1 = xv;
  }
}

// D4 x on a row next to a wall (general reflected weights) as an unevaluated
// pair (S, Er).  Out of line: only the first two and last two rows of a system
// take it, and keeping one copy keeps the unrolled kernel small.
__device__ __noinline__ float2 d4_wall_row(int i, int n, float ah, float al, float bh, float bl, float ch, float cl,
                                           float dh, float dl, float eh, float el) {
  float w[5];
  d4_weights_f(i, n, w);
  const float xs[5] = {ah, bh, ch, dh, eh};
  const float xls[5] = {al, bl, cl, dl, el};
  float S = 0.f, Er = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float p, e, sm, e2;
    two_prod(w[k], xs[k], p, e);
    two_sum(S, p, sm, e2);
    S = sm;
    Er += e + e2 + w[k] * xls[k];
  }
  return make_float2(S, Er);
}

// r = f - (I + sigma D4) x, rounded to FP32, for this thread's rows.  x = xh + xl.
// Float-float residual: f as (fh, fl), sigma as (sgh, sgl).  Rows away from the
// walls use the plain [1, -4, 6, -4, 1] stencil.
__device__ __forceinline__ float residual_row(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                              float dl, float eh, float el, float fhj, float flj, float sgh, float sgl,
                                              int i, int n) {
  float S, Er;
  if (i >= 2 && i + 2 < n) {
    float s1, e1, s2, e2, t, e3, p, e4;
    two_sum(ah, eh, s1, e1);        // x_{i-2} + x_{i+2}
    two_sum(bh, dh, s2, e2);        // x_{i-1} + x_{i+1}
    two_sum(s1, -4.f * s2, t, e3);  // 4 s2 is exact
    two_prod(6.f, ch, p, e4);
    two_sum(t, p, S, Er);
    const float low = fmaf(6.f, cl, fmaf(-4.f, bl + dl, al + el));
    Er = Er + ((e1 - 4.f * e2) + (e3 + e4) + low);
  } else {
    const float2 q = d4_wall_row(i, n, ah, al, bh, bl, ch, cl, dh, dl, eh, el);
    S = q.x;
    Er = q.y;
  }
  float yh, yl;
  fast_two_sum(S, Er, yh, yl);
  float Pp, Pe;  // sigma * y
  two_prod(sgh, yh, Pp, Pe);
  Pe = fmaf(sgh, yl, fmaf(sgl, yh, Pe));
  float a1, a2, b1, b2;
  two_sum(fhj, -ch, a1, a2);
  two_sum(a1, -Pp, b1, b2);
  const float low = ((a2 + b2) + (flj - cl)) - Pe;
  return (i < n) ? (b1 + low) : 0.f;
}

template <int W, int L>
__device__ __forceinline__ void residual_ff(const float (&fh)[L], const float (&fl)[L], const float (&xh)[L],
                                            const float (&xl)[L], float (&r)[L], float sgh, float sgl, int n, int t,
                                            Smem<W>& sm) {
  constexpr int P = 32 * W;
  sm.edge[t][0] = make_float4(xh[0], xh[1], xl[0], xl[1]);
  sm.edge[t][1] = make_float4(xh[L - 2], xh[L - 1], xl[L - 2], xl[L - 1]);
  __syncthreads();
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 prv = (t > 0) ? sm.edge[t - 1][1] : zero;      // rows tL-2, tL-1
  const float4 nxt = (t + 1 < P) ? sm.edge[t + 1][0] : zero;  // rows tL+L, tL+L+1
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float ah = (j >= 2) ? xh[j - 2] : (j == 1 ? prv.y : prv.x);
    const float al = (j >= 2) ? xl[j - 2] : (j == 1 ? prv.w : prv.z);
    const float bh = (j >= 1) ? xh[j - 1] : prv.y;
    const float bl = (j >= 1) ? xl[j - 1] : prv.w;
    const float dh = (j + 1 < L) ? xh[j + 1] : nxt.x;
    const float dl = (j + 1 < L) ? xl[j + 1] : nxt.z;
    const float eh = (j + 2 < L) ? xh[j + 2] : (j + 1 < L ? nxt.x : nxt.y);
    const float el = (j + 2 < L) ? xl[j + 2] : (j + 1 < L ? nxt.z : nxt.w);
    r[j] = residual_row(ah, al, bh, bl, xh[j], xl[j], dh, dl, eh, el, fh[j], fl[j], sgh, sgl, t * L + j, n);
  }
}

// The same residual in native FP64 (the literal reading: FP64 band from sigma,
// FP64 x and f).  xd holds x in FP64 (scaled by 2^-kshift like f).
template <int W, int L>
__device__ __forceinline__ void residual_f64(const double (&fd)[L], const double (&xd)[L], float (&r)[L], double sg,
                                             int n, int t, Smem<W>& sm) {
  constexpr int P = 32 * W;
  double2* ed = reinterpret_cast<double2*>(sm.edge);  // 4 doubles per thread fit in the edge slots
  ed[2 * t] = make_double2(xd[0], xd[1]);
  ed[2 * t + 1] = make_double2(xd[L - 2], xd[L - 1]);
  __syncthreads();
  const double2 zero = make_double2(0.0, 0.0);
  const double2 prv = (t > 0) ? ed[2 * (t - 1) + 1] : zero;
  const double2 nxt = (t + 1 < P) ? ed[2 * (t + 1)] : zero;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int i = t * L + j;
    const double a = (j >= 2) ? xd[j - 2] : (j == 1 ? prv.y : prv.x);
    const double b = (j >= 1) ? xd[j - 1] : prv.y;
    const double d = (j + 1 < L) ? xd[j + 1] : nxt.x;
    const double e = (j + 2 < L) ? xd[j + 2] : (j + 1 < L ? nxt.x : nxt.y);
    double y;
    if (i >= 2 && i + 2 < n) {
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

// epsilon_i = a_i of the hyperdiffusion band: sigma times the weight of x_{i-2}
// in row i, which is 1 for 2 <= i < n (no wall reflection lands there) and 0
// otherwise.
__device__ __forceinline__ float eps_of_row(int i, int n, float sgf) { return (i >= 2 && i < n) ? sgf : 0.f; }

// Load 1/alpha and beta of the thread's rows and rebuild epsilon/alpha,
// beta/alpha, gamma, delta and the two chunk maps.
template <int W, int L>
__device__ __forceinline__ void load_chunk_factors(ChunkFactors<L>& cf, const float4* __restrict__ gq, int t, int n,
                                                   float sgf) {
  constexpr int P = 32 * W;
  float beta[L];
#pragma unroll
  for (int jq = 0; jq < L / 4; ++jq) {
    const float4 qa = __ldg(gq + (jq * 2 + 0) * P + t), qb = __ldg(gq + (jq * 2 + 1) * P + t);
    cf.A[4 * jq] = qa.x; cf.A[4 * jq + 1] = qa.y; cf.A[4 * jq + 2] = qa.z; cf.A[4 * jq + 3] = qa.w;
    beta[4 * jq] = qb.x; beta[4 * jq + 1] = qb.y; beta[4 * jq + 2] = qb.z; beta[4 * jq + 3] = qb.w;
  }
  // beta of the first row of the next thread's chunk (row t L + L)
  const float beta_next = (t + 1 < P) ? __ldg(reinterpret_cast<const float*>(gq + 1 * P + (t + 1))) : 0.f;
  const int i0 = t * L;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int i = i0 + j;
    const float bnext = (j + 1 < L) ? beta[j + 1] : beta_next;
    cf.B[j] = beta[j] * cf.A[j];
    cf.E[j] = eps_of_row(i, n, sgf) * cf.A[j];
    cf.G[j] = bnext * cf.A[j];
    cf.D[j] = eps_of_row(i + 2, n, sgf) * cf.A[j];
  }
  // forward map: acc <- M_j acc with M_j = [[0, 1], [-E_j, -B_j]]
  float f00 = 1.f, f01 = 0.f, f10 = 0.f, f11 = 1.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float n10 = fmaf(-cf.E[j], f00, -cf.B[j] * f10);
    const float n11 = fmaf(-cf.E[j], f01, -cf.B[j] * f11);
    f00 = f10;
    f01 = f11;
    f10 = n10;
    f11 = n11;
  }
  cf.pf = make_float4(f00, f01, f10, f11);
  // backward map: acc <- acc B_j with B_j = [[-G_j, -D_j], [1, 0]], rows ascending
  float t00 = 1.f, t01 = 0.f, t10 = 0.f, t11 = 1.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float n00 = fmaf(-t00, cf.G[j], t01), n01 = -t00 * cf.D[j];
    const float n10 = fmaf(-t10, cf.G[j], t11), n11 = -t10 * cf.D[j];
    t00 = n00;
    t01 = n01;
    t10 = n10;
    t11 = n11;
  }
  cf.pb = make_float4(t00, t01, t10, t11);
}

// One CTA per system: FP32 solve, then up to max_refine refinement steps.
// RES64 selects the FP64 residual (and FP64 accumulation of x) instead of float-float.
// Register budget for up to 8 rows per thread: 512 threads per SM (at most 128
// registers per thread), so that four 128-thread systems share an SM and hide
// each other's barriers.  Longer chunks keep their registers.
template <int W, int L, bool RES64>
__global__ void __launch_bounds__(32 * W, (L <= 8 && 16 / W > 0) ? 16 / W : 1) k_solve32r(int64_t batch, int n, int shared, const float4* __restrict__ fac,
                                                     const double* __restrict__ sigma,
                                                     const float2* __restrict__ sigma2, const double* f, double* x,
                                                     int max_refine, int tol_log2, int vec_io,
                                                     unsigned long long* info) {
  constexpr int P = 32 * W;
  static_assert(L % 4 == 0, "rows per thread must be a multiple of 4");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<W>& sm = *reinterpret_cast<Smem<W>*>(smem_raw);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t s = blockIdx.x;
  if (s >= batch) return;
  const int64_t ms = shared ? 0 : s;
  int phase = 0;

  // ---- loads: factors, right-hand side (all coalesced) ----
  const float2 sgp = __ldg(sigma2 + ms);  // sigma as an FP32 pair, split at factorisation time
  const float sgh = sgp.x, sgl = sgp.y;
  ChunkFactors<L> cf;
  load_chunk_factors<W, L>(cf, fac + ms * (int64_t)(2 * P * L / 4), t, n, sgh);
  const double* fs = f + s * (int64_t)n;
  const int i0 = t * L;
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

  // ---- per-system power-of-two scale: the largest |f| maps just below 1 ----
  int emax = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const unsigned top = (unsigned)((unsigned long long)__double_as_longlong(fv[j]) >> 32);
    emax = max(emax, (int)((top >> 20) & 0x7ffu));
  }
  emax = block_max_i<W>(emax, lane, warp, sm.redi);
  const int kshift = emax - 1022;

  float v[L], xh[L], xl[L];
  float fh[L], fl[L];
#pragma unroll
  for (int j = 0; j < L; ++j) split_scaled(fv[j], kshift, fh[j], fl[j]);
#pragma unroll
  for (int j = 0; j < L; ++j) v[j] = fh[j];
  int steps = 0;
  bool stalled = false;
  if (RES64) {
    // x kept in FP64 (scaled by 2^-kshift); f in FP64 scaled the same way
    double xd[L], fd[L];
    const double scale = ldexp(1.0, -kshift);
    const double sg = sigma[ms];
#pragma unroll
    for (int j = 0; j < L; ++j) fd[j] = fv[j] * scale;
    float prev = INFINITY;
    const float tol = ldexpf(1.0f, -tol_log2);
#pragma unroll 1
    for (int it = 0; it <= max_refine; ++it) {
      if (it > 0) residual_f64<W, L>(fd, xd, v, sg, n, t, sm);
      cta_solve32<W, L>(v, cf, lane, warp, sm, phase);
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
        dmax = block_max<W>(dmax, lane, warp, sm.red[phase & 3]);
        xmax = block_max<W>(xmax, lane, warp, sm.red[phase & 3] + W);
        ++phase;
        if (dmax <= tol * xmax) break;
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
    float prev = INFINITY;
    const float tol = ldexpf(1.0f, -tol_log2);
    // it = 0 solves for f (its FP32 part); every later pass solves for the
    // float-float residual of the current x and adds the correction.  One
    // solve call site keeps the unrolled kernel compact.
#pragma unroll 1
    for (int it = 0; it <= max_refine; ++it) {
      if (it > 0) residual_ff<W, L>(fh, fl, xh, xl, v, sgh, sgl, n, t, sm);
      cta_solve32<W, L>(v, cf, lane, warp, sm, phase);
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
        dmax = block_max<W>(dmax, lane, warp, sm.red[phase & 3]);
        xmax = block_max<W>(xmax, lane, warp, sm.red[phase & 3] + W);
        ++phase;
        if (dmax <= tol * xmax) break;
        if (it > 1 && dmax > 0.5f * prev) {
          stalled = true;
          break;
        }
        prev = dmax;
      }
    }
#pragma unroll
    for (int j = 0; j < L; ++j) fv[j] = f2d_shift(xh[j], kshift) + f2d_shift(xl[j], kshift);
  }
  if (t == 0) {
    if (steps > 0) atomicMax(info + 1, (unsigned long long)steps);
    if (stalled) atomicOr(info + 2, 1ull);
  }
  // ---- store x (a thread's rows are contiguous) ----
  double* xs = x + s * (int64_t)n;
  if (vec_io && i0 + L <= n) {
#pragma unroll
    for (int j = 0; j < L; j += 2) *reinterpret_cast<double2*>(xs + i0 + j) = make_double2(fv[j], fv[j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j)
      if (i0 + j < n) xs[i0 + j] = fv[j];
  }
}

// Factor A = I + sigma D4 of one system per thread in FP64 (Sec. 2.4,
// factorisation steps 1-14) and store 1/alpha and beta rounded to FP32 in the
// CTA-per-system layout: float4 ((s * L/4 + j/4) * 2 + p) * P + t holds rows
// t L + 4 (j/4) .. + 3 of plane p (0: 1/alpha, 1: beta).
__global__ void k_factor32(DevPlan P, int n, int Pt, int L, const double* __restrict__ sigma, float* __restrict__ fac,
                           float2* __restrict__ sigma2) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nsys = P.shared ? 1 : P.batch;
  if (s >= nsys) return;
  const double sg = sigma[s];
  {
    const float hi = __double2float_rn(sg);
    sigma2[s] = make_float2(hi, __double2float_rn(sg - (double)hi));
  }
  float* F = fac + s * (int64_t)2 * Pt * L;
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;
  bool failed = false;
  const int rows = Pt * L;
  for (int i = 0; i < rows; ++i) {
    float ainv = 1.f, bt = 0.f;
    if (i < n && !failed) {
      float w[5];
      d4_weights_f(i, n, w);
      const double ar = (i >= 2) ? sg * w[0] : 0.0;
      const double br = (i >= 1) ? sg * w[1] : 0.0;
      const double cr = 1.0 + sg * w[2];
      const double dr = (i + 1 < n) ? sg * w[3] : 0.0;
      const double er = (i + 2 < n) ? sg * w[4] : 0.0;
      const double beta = br - ar * gam2;
      const double alpha = cr - ar * del2 - beta * gam1;
      if (!(alpha != 0.0) || !isfinite(alpha)) {
        const unsigned long long key = ((unsigned long long)s << 32) | (unsigned long long)(uint32_t)i;
        atomicMin(P.info, key);
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
    const int t = i / L, j = i - t * L;
    const int64_t base = ((int64_t)(j / 4) * 2) * Pt * 4 + (int64_t)t * 4 + (j & 3);
    F[base] = ainv;
    F[base + (int64_t)Pt * 4] = bt;
  }
}

template <int W, int L, bool RES64>
cudaError_t launch_solve32r_WL(const DevPlan& P, const F32Factors& F, const double* sigma, int n, const double* f,
                               double* x, int max_refine, int tol_log2, cudaStream_t st) {
  const int vec = ((((uintptr_t)f) | ((uintptr_t)x)) % 16 == 0) && (n % 2 == 0);
  constexpr size_t smem = sizeof(Smem<W>);
  static bool attr = false;  // once per process; not a stream operation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_solve32r<W, L, RES64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_solve32r<W, L, RES64><<<(unsigned)P.batch, 32 * W, smem, st>>>(P.batch, n, P.shared,
                                                                 reinterpret_cast<const float4*>(F.fac), sigma,
                                                                 reinterpret_cast<const float2*>(F.sigma2), f, x,
                                                                 max_refine, tol_log2, vec, P.info);
  return cudaGetLastError();
}

template <bool RES64>
cudaError_t dispatch32(const DevPlan& P, const F32Factors& F, const double* sigma, int n, const double* f, double* x,
                       int max_refine, int tol_log2, cudaStream_t st) {
#define PENT_CASE(W_, L_) \
  if (F.W == W_ && F.L == L_) return launch_solve32r_WL<W_, L_, RES64>(P, F, sigma, n, f, x, max_refine, tol_log2, st);
  PENT_CASE(1, 4) PENT_CASE(1, 8) PENT_CASE(1, 16)
  PENT_CASE(2, 4) PENT_CASE(2, 8) PENT_CASE(2, 16)
  PENT_CASE(4, 4) PENT_CASE(4, 8) PENT_CASE(4, 16)
  PENT_CASE(8, 4) PENT_CASE(8, 8) PENT_CASE(8, 16)
  PENT_CASE(16, 8)
#undef PENT_CASE
  return cudaErrorInvalidValue;
}

}  // namespace

bool f32_shape_supported(int W, int L) {
  static const int shapes[][2] = {{1, 4}, {1, 8}, {1, 16}, {2, 4}, {2, 8}, {2, 16}, {4, 4},
                                  {4, 8}, {4, 16}, {8, 4}, {8, 8}, {8, 16}, {16, 8}};
  for (const auto& sh : shapes)
    if (sh[0] == W && sh[1] == L) return true;
  return false;
}

cudaError_t launch_factor32(const DevPlan& P, const double* sigma, F32Factors F, int n, cudaStream_t st) {
  const int64_t nsys = P.shared ? 1 : P.batch;
  const int block = 128;
  k_factor32<<<(unsigned)((nsys + block - 1) / block), block, 0, st>>>(P, n, 32 * F.W, F.L, sigma, F.fac,
                                                                       reinterpret_cast<float2*>(F.sigma2));
  return cudaGetLastError();
}

cudaError_t launch_solve32r(const DevPlan& P, F32Factors F, const double* sigma, int n, const double* f, double* x,
                            int max_refine, int residual_f64, int tol_log2, cudaStream_t st) {
  return residual_f64 ? dispatch32<true>(P, F, sigma, n, f, x, max_refine, tol_log2, st)
                      : dispatch32<false>(P, F, sigma, n, f, x, max_refine, tol_log2, st);
}

}  // namespace pent
