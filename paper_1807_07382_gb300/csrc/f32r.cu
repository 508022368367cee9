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
// values as an affine map.  The thread runs its chunk from a zero state to get
// the affine part; the maps are composed by a Kogge-Stone shuffle scan in each
// warp, a short carry across warps and, in a cluster, a carry across CTAs read
// through distributed shared memory; then every thread reruns its chunk from
// the true entering state.  The factors are read from HBM once per call
// and reused by every substitution of every refinement step.
//
// The hyperdiffusion matrices are symmetric, so A = L D^{-1} L^T with D the
// diagonal alpha of L: R = D^{-1} L^T, gamma_i = beta_{i+1} / alpha_i and
// delta_i = epsilon_{i+2} / alpha_i, and epsilon_i = a_i is sigma times a
// stencil weight.  Only 1/alpha_i and beta_i are stored (8 bytes per row in
// FP32); epsilon, gamma, delta and the chunks' 2x2 transfer maps are rebuilt in
// registers, trading FP32 arithmetic for HBM bytes.
#include <cooperative_groups.h>

#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace cg = cooperative_groups;

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

// Weights of the no-flux fourth difference on row i (n rows, 0 <= i < n),
// reflected about the cell-centred walls; w[k] multiplies x_{i+k-2}.  Small
// integers.  For rows inside the system every reflected column lies within
// i-2 .. i+2; the bounds test keeps the local array safe for any argument.
__device__ __forceinline__ void d4_weights_f(int i, int n, float w[5]) {
  const float st[5] = {1.f, -4.f, 6.f, -4.f, 1.f};
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    int j = i + k - 2;
    while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
    const int at = j - i + 2;  // within 0..4 for every row 0 <= i < n
    if (at >= 0 && at < 5) w[at] += st[k];
  }
}

// ---------------------------------------------------------------- block / cluster scans

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

__device__ __forceinline__ void apply(const float4 m, const float4 b, float& c0, float& c1) {
  const float n0 = fmaf(m.x, c0, fmaf(m.y, c1, b.x));
  const float n1 = fmaf(m.z, c0, fmaf(m.w, c1, b.y));
  c0 = n0;
  c1 = n1;
}

// Entering state of this thread's chunk for a sweep through the system's chunks.
// FWD: chunks in increasing thread order; otherwise decreasing.  `a` is this
// chunk's map (linear part from the factors, affine part from a zero-state
// pass); the system is entered with state 0.  The Kogge-Stone levels stop as
// soon as every lane's window either reaches the warp's first chunk or
// composes to a negligible linear part (later levels would only add terms
// multiplied by it).  sh: 2 W + 2 float4 (warp totals, then the CTA total).
template <bool FWD>
__device__ __forceinline__ void scan_entry(Aff a, int lane, int warp, int W, int C, int rank, float4* sh, float& e0,
                                           float& e1) {
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
  if (W > 1 || C > 1) {
    if (FWD ? (lane == 31) : (lane == 0)) {
      sh[2 * warp] = make_float4(a.a, a.b, a.c, a.d);
      sh[2 * warp + 1] = make_float4(a.u, a.v, 0.f, 0.f);
    }
    __syncthreads();
    if (C > 1) {
      if (threadIdx.x == 0) {  // the CTA's total map, published for the other CTAs of the cluster
        float4 tm = make_float4(1.f, 0.f, 0.f, 1.f), tb = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < W; ++k) {
          const int w = FWD ? k : W - 1 - k;
          const Aff L{sh[2 * w].x, sh[2 * w].y, sh[2 * w].z, sh[2 * w].w, sh[2 * w + 1].x, sh[2 * w + 1].y};
          const Aff t = compose(L, Aff{tm.x, tm.y, tm.z, tm.w, tb.x, tb.y});
          tm = make_float4(t.a, t.b, t.c, t.d);
          tb = make_float4(t.u, t.v, 0.f, 0.f);
        }
        sh[2 * W] = tm;
        sh[2 * W + 1] = tb;
      }
      cg::this_cluster().sync();
      if (FWD) {
        for (int r = 0; r < rank; ++r) {
          const float4* q = remote(sh, r);
          apply(q[2 * W], q[2 * W + 1], c0, c1);
        }
      } else {
        for (int r = C - 1; r > rank; --r) {
          const float4* q = remote(sh, r);
          apply(q[2 * W], q[2 * W + 1], c0, c1);
        }
      }
    }
    if (FWD) {
      for (int w = 0; w < warp; ++w) apply(sh[2 * w], sh[2 * w + 1], c0, c1);
    } else {
      for (int w = W - 1; w > warp; --w) apply(sh[2 * w], sh[2 * w + 1], c0, c1);
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

// Shared scratch of one CTA (dynamic; W is a launch parameter).  Scan and
// reduction slots rotate through four buffers, so one barrier per scan
// separates every write from the reads of the same buffer, in this CTA and in
// the other CTAs of a cluster.
struct SmemView {
  float4* scan;  // [4][2W + 2]
  float4* edge;  // [P][2]: first two rows (hi, lo), last two rows (hi, lo)
  float* red;    // [4][W + 1]
  int* redi;     // [W + 1]
};

__host__ __device__ inline size_t smem_bytes(int W) {
  return sizeof(float4) * (size_t)(4 * (2 * W + 2) + 2 * 32 * W) + sizeof(float) * (size_t)(4 * (W + 1)) +
         sizeof(int) * (size_t)(W + 1);
}

__device__ __forceinline__ SmemView smem_view(unsigned char* base, int W) {
  SmemView v;
  v.scan = reinterpret_cast<float4*>(base);
  v.edge = v.scan + 4 * (2 * W + 2);
  v.red = reinterpret_cast<float*>(v.edge + 2 * 32 * W);
  v.redi = reinterpret_cast<int*>(v.red + 4 * (W + 1));
  return v;
}

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

struct Ctx {
  int lane, warp, W, C, rank;
  int phase;
};

// In place v <- A^{-1} v (FP32): forward L g = v, then back R x = g.
template <int L>
__device__ __forceinline__ void cta_solve32(float (&v)[L], const ChunkFactors<L>& cf, Ctx& cx, const SmemView& sm) {
  float p2 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float g = fmaf(-cf.B[j], p1, fmaf(-cf.E[j], p2, cf.A[j] * v[j]));
    p2 = p1;
    p1 = g;
  }
  float e0, e1;
  scan_entry<true>(Aff{cf.pf.x, cf.pf.y, cf.pf.z, cf.pf.w, p2, p1}, cx.lane, cx.warp, cx.W, cx.C, cx.rank,
                   sm.scan + (cx.phase++ & 3) * (2 * cx.W + 2), e0, e1);
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
  scan_entry<false>(Aff{cf.pb.x, cf.pb.y, cf.pb.z, cf.pb.w, s1, s2}, cx.lane, cx.warp, cx.W, cx.C, cx.rank,
                    sm.scan + (cx.phase++ & 3) * (2 * cx.W + 2), e0, e1);
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

// r = f - (I + sigma D4) x for one row, in float-float (x = xh + xl, f = fh + fl,
// sigma = sgh + sgl), rounded to FP32.  Rows away from the walls use the plain
// [1, -4, 6, -4, 1] stencil.
__device__ __forceinline__ float residual_row(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                              float dl, float eh, float el, float fhj, float flj, float sgh, float sgl,
                                              int i, int n) {
  if (i >= n) return 0.f;  // padding row past the end of the system
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
  return b1 + low;
}

// The neighbouring rows of this thread's chunk: the last two rows of the
// previous chunk and the first two of the next, across warps through shared
// memory and across CTAs of a cluster through distributed shared memory.
template <int L>
__device__ __forceinline__ void exchange_edges(float4 own_first, float4 own_last, int t, int P, const Ctx& cx,
                                               const SmemView& sm, float4& prv, float4& nxt) {
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

template <int L>
__device__ __forceinline__ void residual_ff(const float (&fh)[L], const float (&fl)[L], const float (&xh)[L],
                                            const float (&xl)[L], float (&r)[L], float sgh, float sgl, int n, int t,
                                            int tg, int P, const Ctx& cx, const SmemView& sm) {
  float4 prv, nxt;
  exchange_edges<L>(make_float4(xh[0], xh[1], xl[0], xl[1]), make_float4(xh[L - 2], xh[L - 1], xl[L - 2], xl[L - 1]),
                    t, P, cx, sm, prv, nxt);
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
    r[j] = residual_row(ah, al, bh, bl, xh[j], xl[j], dh, dl, eh, el, fh[j], fl[j], sgh, sgl, tg * L + j, n);
  }
}

// The same residual in native FP64 (the literal reading: FP64 band from sigma,
// FP64 x and f).  xd holds x in FP64 (scaled by 2^-kshift like f).  The edge
// slots carry the neighbouring rows as double pairs.
template <int L>
__device__ __forceinline__ void residual_f64(const double (&fd)[L], const double (&xd)[L], float (&r)[L], double sg,
                                             int n, int t, int tg, int P, const Ctx& cx, const SmemView& sm) {
  float4 pf4, nf4;
  const double2 f2 = make_double2(xd[0], xd[1]), l2 = make_double2(xd[L - 2], xd[L - 1]);
  exchange_edges<L>(*reinterpret_cast<const float4*>(&f2), *reinterpret_cast<const float4*>(&l2), t, P, cx, sm, pf4,
                    nf4);
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

// epsilon_i = a_i of the hyperdiffusion band: sigma times the weight of x_{i-2}
// in row i, which is 1 for 2 <= i < n (no wall reflection lands there) and 0
// otherwise.
__device__ __forceinline__ float eps_of_row(int i, int n, float sgf) { return (i >= 2 && i < n) ? sgf : 0.f; }

// Load 1/alpha and beta of the thread's rows and rebuild epsilon/alpha,
// beta/alpha, gamma, delta and the two chunk maps.  gq: the system's factor
// block; PT threads per system; tg this thread's index in the system.
template <int L>
__device__ __forceinline__ void load_chunk_factors(ChunkFactors<L>& cf, const float4* __restrict__ gq, int tg, int PT,
                                                   int n, float sgf) {
  float beta[L];
#pragma unroll
  for (int jq = 0; jq < L / 4; ++jq) {
    const float4 qa = __ldg(gq + (int64_t)(jq * 2 + 0) * PT + tg), qb = __ldg(gq + (int64_t)(jq * 2 + 1) * PT + tg);
    cf.A[4 * jq] = qa.x; cf.A[4 * jq + 1] = qa.y; cf.A[4 * jq + 2] = qa.z; cf.A[4 * jq + 3] = qa.w;
    beta[4 * jq] = qb.x; beta[4 * jq + 1] = qb.y; beta[4 * jq + 2] = qb.z; beta[4 * jq + 3] = qb.w;
  }
  // beta of the first row of the next thread's chunk (row tg L + L)
  const float beta_next = (tg + 1 < PT) ? __ldg(reinterpret_cast<const float*>(gq + (int64_t)PT + (tg + 1))) : 0.f;
  const int i0 = tg * L;
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

// One CTA (or one cluster of C CTAs) per system: FP32 solve, then up to
// max_refine refinement steps.  RES64 selects the FP64 residual (and FP64
// accumulation of x) instead of float-float.  Register budget: 512 threads per
// SM (at most 128 registers per thread), so up to four 128-thread systems share
// an SM and hide each other's barriers.
// WT > 0 fixes the warp count at compile time (the common one-CTA shapes);
// WT = 0 takes it from `Wrt`.  CL enables the cluster paths (C = Crt CTAs per
// system), otherwise C = 1.
constexpr int min_blocks(int L, int WT) { return WT > 0 ? ((L <= 8 && 16 / WT > 0) ? 16 / WT : 1) : 1; }

template <int L, int WT, bool CL, bool RES64>
__global__ void __launch_bounds__(WT > 0 ? 32 * WT : 512, min_blocks(L, WT))
    k_solve32r(F32Tables T, const int32_t* __restrict__ sys, int Wrt, int Crt, int shared, const double* f, double* x,
               int max_refine, int tol_log2, int vec_io) {
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
  ChunkFactors<L> cf;
  load_chunk_factors<L>(cf, reinterpret_cast<const float4*>(T.fac) + T.foff[ms], tg, PT, n, sgh);
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

  // ---- per-system power-of-two scale: the largest |f| maps just below 1 ----
  int emax = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const unsigned top = (unsigned)((unsigned long long)__double_as_longlong(fv[j]) >> 32);
    emax = max(emax, (int)((top >> 20) & 0x7ffu));
  }
  emax = system_max<int>(emax, cx.lane, cx.warp, W, C, sm.redi);
  const int kshift = emax - 1022;

  float v[L], xh[L], xl[L];
  float fh[L], fl[L];
#pragma unroll
  for (int j = 0; j < L; ++j) split_scaled(fv[j], kshift, fh[j], fl[j]);
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
      if (it > 0) residual_f64<L>(fd, xd, v, sg, n, t, tg, P, cx, sm);
      cta_solve32<L>(v, cf, cx, sm);
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
        float* rs = sm.red + (cx.phase & 3) * (W + 1);
        ++cx.phase;
        dmax = system_max<float>(dmax, cx.lane, cx.warp, W, C, rs);
        float* rs2 = sm.red + (cx.phase & 3) * (W + 1);
        ++cx.phase;
        xmax = system_max<float>(xmax, cx.lane, cx.warp, W, C, rs2);
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
    // it = 0 solves for f (its FP32 part); every later pass solves for the
    // float-float residual of the current x and adds the correction.  One
    // solve call site keeps the unrolled kernel compact.
#pragma unroll 1
    for (int it = 0; it <= max_refine; ++it) {
      if (it > 0) residual_ff<L>(fh, fl, xh, xl, v, sgh, sgl, n, t, tg, P, cx, sm);
      cta_solve32<L>(v, cf, cx, sm);
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
        float* rs = sm.red + (cx.phase & 3) * (W + 1);
        ++cx.phase;
        dmax = system_max<float>(dmax, cx.lane, cx.warp, W, C, rs);
        float* rs2 = sm.red + (cx.phase & 3) * (W + 1);
        ++cx.phase;
        xmax = system_max<float>(xmax, cx.lane, cx.warp, W, C, rs2);
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

template <int L, int WT, bool CL, bool RES64>
cudaError_t launch_bucket(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                          double* x, int max_refine, int tol_log2, cudaStream_t st) {
  const int vec = ((((uintptr_t)f) | ((uintptr_t)x)) % 16 == 0) && b.even_offsets;
  const size_t smem = smem_bytes(b.W);
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
  return cudaLaunchKernelEx(&cfg, k_solve32r<L, WT, CL, RES64>, T, sys + b.first, b.W, b.C, shared, f, x, max_refine,
                            tol_log2, vec);
}

template <int L, bool RES64>
cudaError_t dispatch_bucket(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                            double* x, int max_refine, int tol_log2, cudaStream_t st) {
  if (b.C > 1) return launch_bucket<L, 0, true, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
  if (!RES64) {
    switch (b.W) {
      case 1: return launch_bucket<L, 1, false, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
      case 2: return launch_bucket<L, 2, false, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
      case 4: return launch_bucket<L, 4, false, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
      case 8: return launch_bucket<L, 8, false, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
      case 16: return launch_bucket<L, 16, false, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
      default: break;
    }
  }
  return launch_bucket<L, 0, false, RES64>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
}

}  // namespace

cudaError_t launch_factor32(const F32Tables& T, const int32_t* shape, int64_t nsys, const double* sigma,
                            cudaStream_t st) {
  const int block = 128;
  k_factor32<<<(unsigned)((nsys + block - 1) / block), block, 0, st>>>(T, nsys, shape, sigma);
  return cudaGetLastError();
}

cudaError_t launch_solve32r(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                            double* x, int max_refine, int residual_f64, int tol_log2, cudaStream_t st) {
  if (b.count == 0) return cudaSuccess;
  if (b.L == 4) return residual_f64 ? dispatch_bucket<4, true>(T, sys, b, shared, f, x, max_refine, tol_log2, st)
                                    : dispatch_bucket<4, false>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
  if (b.L == 8) return residual_f64 ? dispatch_bucket<8, true>(T, sys, b, shared, f, x, max_refine, tol_log2, st)
                                    : dispatch_bucket<8, false>(T, sys, b, shared, f, x, max_refine, tol_log2, st);
  return cudaErrorInvalidValue;
}

}  // namespace pent
