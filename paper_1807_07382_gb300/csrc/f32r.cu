// FP32 substitution with iterative refinement, one warp per system.
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
// One warp owns one system of n <= 32 L rows: lane t holds rows t L .. t L + L - 1
// in registers.  Each substitution (Sec. 2.4: L g = f, then R x = g) is a
// second-order linear recurrence, so a lane's chunk acts on the two carried
// values as an affine map.  The lane runs its chunk from a zero state to get
// the affine part, the warp composes the maps with a Kogge-Stone shuffle scan
// (the 2x2 linear parts of the chunks are precomputed at factorisation time,
// because they depend on the factors only), and every lane reruns its chunk
// from the true entering state.  The system's factors (20 bytes per row) are
// staged once in shared memory and reused by every substitution of every
// refinement step, so a refined solve reads its factors from HBM once.
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace pent {
namespace {

// ---------------------------------------------------------------- async copies (sm_80+ cp.async)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

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

// Exact v * 2^k as a double, by moving v's exponent and mantissa bit fields.
__device__ __forceinline__ double f2d_shift(float v, int k) {
  const unsigned u = __float_as_uint(v);
  const unsigned a = u & 0x7fffffffu;
  if (a == 0u) return 0.0;
  const int e = (int)(a >> 23);
  const int de = e + 896 + k;
  if (e == 0 || e == 255 || de < 1 || de > 2046) return ldexp((double)v, k);  // rare: subnormal / out of range
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

// ---------------------------------------------------------------- chunked warp substitution

// In place v <- A^{-1} v for the warp's system in FP32 (forward L g = v, back R x = g).
// sf: the system's factor planes in shared memory, slot j*32 + lane.
template <int L>
__device__ __forceinline__ void warp_solve32(float (&v)[L], const float* __restrict__ sf, const float4 pf,
                                             const float4 pb, int lane) {
  const float* A = sf;
  const float* B = sf + 32 * L;
  const float* E = sf + 64 * L;
  const float* G = sf + 96 * L;
  const float* D = sf + 128 * L;
  // forward, pass 1: chunk from a zero entering state -> affine part (p2, p1)
  float p2 = 0.f, p1 = 0.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int o = j * 32 + lane;
    const float g = fmaf(-B[o], p1, fmaf(-E[o], p2, A[o] * v[j]));
    p2 = p1;
    p1 = g;
  }
  // inclusive scan of affine maps (entering (g_{i-2}, g_{i-1}) -> leaving), earlier lanes first
  float m00 = pf.x, m01 = pf.y, m10 = pf.z, m11 = pf.w, b0 = p2, b1 = p1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float o00 = __shfl_up_sync(0xffffffffu, m00, d), o01 = __shfl_up_sync(0xffffffffu, m01, d);
    const float o10 = __shfl_up_sync(0xffffffffu, m10, d), o11 = __shfl_up_sync(0xffffffffu, m11, d);
    const float ob0 = __shfl_up_sync(0xffffffffu, b0, d), ob1 = __shfl_up_sync(0xffffffffu, b1, d);
    if (lane >= d) {
      const float n00 = fmaf(m00, o00, m01 * o10), n01 = fmaf(m00, o01, m01 * o11);
      const float n10 = fmaf(m10, o00, m11 * o10), n11 = fmaf(m10, o01, m11 * o11);
      const float nb0 = fmaf(m00, ob0, fmaf(m01, ob1, b0));
      const float nb1 = fmaf(m10, ob0, fmaf(m11, ob1, b1));
      m00 = n00; m01 = n01; m10 = n10; m11 = n11; b0 = nb0; b1 = nb1;
    }
  }
  p2 = __shfl_up_sync(0xffffffffu, b0, 1);
  p1 = __shfl_up_sync(0xffffffffu, b1, 1);
  if (lane == 0) p2 = p1 = 0.f;
  // forward, pass 2 from the true entering state
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int o = j * 32 + lane;
    const float g = fmaf(-B[o], p1, fmaf(-E[o], p2, A[o] * v[j]));
    v[j] = g;
    p2 = p1;
    p1 = g;
  }
  // back, pass 1: descending from a zero entering state (x_{i+1}, x_{i+2})
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const int o = j * 32 + lane;
    const float xv = fmaf(-G[o], s1, fmaf(-D[o], s2, v[j]));
    s2 = s1;
    s1 = xv;
  }
  m00 = pb.x; m01 = pb.y; m10 = pb.z; m11 = pb.w; b0 = s1; b1 = s2;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float o00 = __shfl_down_sync(0xffffffffu, m00, d), o01 = __shfl_down_sync(0xffffffffu, m01, d);
    const float o10 = __shfl_down_sync(0xffffffffu, m10, d), o11 = __shfl_down_sync(0xffffffffu, m11, d);
    const float ob0 = __shfl_down_sync(0xffffffffu, b0, d), ob1 = __shfl_down_sync(0xffffffffu, b1, d);
    if (lane + d < 32) {
      const float n00 = fmaf(m00, o00, m01 * o10), n01 = fmaf(m00, o01, m01 * o11);
      const float n10 = fmaf(m10, o00, m11 * o10), n11 = fmaf(m10, o01, m11 * o11);
      const float nb0 = fmaf(m00, ob0, fmaf(m01, ob1, b0));
      const float nb1 = fmaf(m10, ob0, fmaf(m11, ob1, b1));
      m00 = n00; m01 = n01; m10 = n10; m11 = n11; b0 = nb0; b1 = nb1;
    }
  }
  s1 = __shfl_down_sync(0xffffffffu, b0, 1);
  s2 = __shfl_down_sync(0xffffffffu, b1, 1);
  if (lane == 31) s1 = s2 = 0.f;
#pragma unroll
  for (int j = L - 1; j >= 0; --j) {
    const int o = j * 32 + lane;
    const float xv = fmaf(-G[o], s1, fmaf(-D[o], s2, v[j]));
    v[j] = xv;
    s2 = s1;
    s1 = xv;
  }
}

// r = f - (I + sigma D4) x in float-float, rounded to FP32.  f is read from the
// shared-memory copy (FP64) and split on the fly; x = xh + xl; the two rows on
// each side of a lane's chunk come from the neighbouring lanes.
template <int L>
__device__ __forceinline__ void residual_hyperdiff(const double* __restrict__ sfx, int kshift, const float (&xh)[L],
                                                   const float (&xl)[L], float (&r)[L], float sgh, float sgl, int n,
                                                   int lane) {
  float m2h = __shfl_up_sync(0xffffffffu, xh[L - 2], 1), m1h = __shfl_up_sync(0xffffffffu, xh[L - 1], 1);
  float m2l = __shfl_up_sync(0xffffffffu, xl[L - 2], 1), m1l = __shfl_up_sync(0xffffffffu, xl[L - 1], 1);
  float p1h = __shfl_down_sync(0xffffffffu, xh[0], 1), p2h = __shfl_down_sync(0xffffffffu, xh[1], 1);
  float p1l = __shfl_down_sync(0xffffffffu, xl[0], 1), p2l = __shfl_down_sync(0xffffffffu, xl[1], 1);
  if (lane == 0) m2h = m1h = m2l = m1l = 0.f;
  if (lane == 31) p1h = p2h = p1l = p2l = 0.f;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int i = lane * L + j;
    const float ah = (j >= 2) ? xh[j - 2] : (j == 1 ? m1h : m2h);
    const float al = (j >= 2) ? xl[j - 2] : (j == 1 ? m1l : m2l);
    const float bh = (j >= 1) ? xh[j - 1] : m1h;
    const float bl = (j >= 1) ? xl[j - 1] : m1l;
    const float dh = (j + 1 < L) ? xh[j + 1] : p1h;
    const float dl = (j + 1 < L) ? xl[j + 1] : p1l;
    const float eh = (j + 2 < L) ? xh[j + 2] : (j + 1 < L ? p1h : p2h);
    const float el = (j + 2 < L) ? xl[j + 2] : (j + 1 < L ? p1l : p2l);
    const float ch = xh[j], cl = xl[j];
    float S, Er;  // D4 x as S + Er
    if (i >= 2 && i + 2 < n) {
      float s1, e1, s2, e2, t, e3, p, e4;
      two_sum(ah, eh, s1, e1);           // x_{i-2} + x_{i+2}
      two_sum(bh, dh, s2, e2);           // x_{i-1} + x_{i+1}
      two_sum(s1, -4.f * s2, t, e3);     // 4 s2 is exact
      two_prod(6.f, ch, p, e4);
      two_sum(t, p, S, Er);
      const float low = fmaf(6.f, cl, fmaf(-4.f, bl + dl, al + el));
      Er = Er + (e1 - 4.f * e2 + e3 + e4 + low);
    } else {
      float w[5];
      d4_weights_f(i, n, w);
      const float xs[5] = {ah, bh, ch, dh, eh};
      const float xls[5] = {al, bl, cl, dl, el};
      S = 0.f;
      Er = 0.f;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        float p, e, s, e2;
        two_prod(w[k], xs[k], p, e);
        two_sum(S, p, s, e2);
        S = s;
        Er += e + e2 + w[k] * xls[k];
      }
    }
    float yh, yl;
    fast_two_sum(S, Er, yh, yl);
    // sigma * y
    float P, Pe;
    two_prod(sgh, yh, P, Pe);
    Pe = fmaf(sgh, yl, fmaf(sgl, yh, Pe));
    // f - x - sigma D4 x
    float fh, fl;
    split_scaled(sfx[j * 33 + lane], kshift, fh, fl);
    float a1, a2, b1, b2;
    two_sum(fh, -ch, a1, a2);
    two_sum(a1, -P, b1, b2);
    const float low = ((a2 + b2) + (fl - cl)) - Pe;
    r[j] = (i < n) ? (b1 + low) : 0.f;
  }
}

// One warp per system: FP32 solve, then up to max_refine float-float refinement steps.
template <int L>
__global__ void __launch_bounds__(32 * 8) k_solve32r(int64_t batch, int n, int shared, const float* __restrict__ fac,
                                                     const float* __restrict__ phi, const double* __restrict__ sigma,
                                                     const double* f, double* x, int max_refine, int tol_log2,
                                                     unsigned long long* info) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kFacFloats = 5 * 32 * L;
  constexpr int kBytesPerWarp = kFacFloats * 4 + L * 33 * 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
  if (s >= batch) return;
  float* sf = reinterpret_cast<float*>(smem + (size_t)warp * kBytesPerWarp);
  double* sx = reinterpret_cast<double*>(sf + kFacFloats);
  const int64_t ms = shared ? 0 : s;
  const float* gfac = fac + ms * kFacFloats;
#pragma unroll 4
  for (int c = lane; c < kFacFloats / 4; c += 32) cp_async16(sf + 4 * c, gfac + 4 * c);
  const double* gf = f + s * (int64_t)n;
#pragma unroll 4
  for (int m = 0; m < L; ++m) {
    const int i = 32 * m + lane;
    const int t = i / L, j = i - t * L;
    if (i < n)
      cp_async8(sx + j * 33 + t, gf + i);
    else
      sx[j * 33 + t] = 0.0;
  }
  const float4* gphi = reinterpret_cast<const float4*>(phi + (ms * 32 + lane) * 8);
  const float4 pf = __ldg(gphi), pb = __ldg(gphi + 1);
  const double sg = sigma[ms];
  const float sgh = __double2float_rn(sg);
  const float sgl = __double2float_rn(sg - (double)sgh);
  cp_async_wait_all();
  __syncwarp();

  // per-system power-of-two scale: largest |f| maps just below 1
  int emax = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const unsigned top = (unsigned)((unsigned long long)__double_as_longlong(sx[j * 33 + lane]) >> 32);
    emax = max(emax, (int)((top >> 20) & 0x7ffu));
  }
  emax = warp_max_i(emax);
  const int kshift = emax - 1022;

  float xh[L], xl[L], v[L];
#pragma unroll
  for (int j = 0; j < L; ++j) {
    float lo;
    split_scaled(sx[j * 33 + lane], kshift, v[j], lo);
  }
  warp_solve32<L>(v, sf, pf, pb, lane);
#pragma unroll
  for (int j = 0; j < L; ++j) {
    xh[j] = v[j];
    xl[j] = 0.f;
  }
  int steps = 0;
  float prev = INFINITY;
  const float tol = ldexpf(1.0f, -tol_log2);
  bool stalled = false;
  for (int it = 0; it < max_refine; ++it) {
    residual_hyperdiff<L>(sx, kshift, xh, xl, v, sgh, sgl, n, lane);
    warp_solve32<L>(v, sf, pf, pb, lane);
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
    dmax = warp_max(dmax);
    xmax = warp_max(xmax);
    steps = it + 1;
    if (dmax <= tol * xmax) break;
    if (it > 0 && dmax > 0.5f * prev) {
      stalled = true;
      break;
    }
    prev = dmax;
  }
  if (lane == 0) {
    if (steps > 0) atomicMax(info + 1, (unsigned long long)steps);
    if (stalled) atomicOr(info + 2, 1ull);
  }
  // x = 2^k (xh + xl) in FP64, transposed through shared memory for coalesced stores
  __syncwarp();
#pragma unroll
  for (int j = 0; j < L; ++j) sx[j * 33 + lane] = f2d_shift(xh[j], kshift) + f2d_shift(xl[j], kshift);
  __syncwarp();
  double* gx = x + s * (int64_t)n;
#pragma unroll 4
  for (int m = 0; m < L; ++m) {
    const int i = 32 * m + lane;
    const int t = i / L, j = i - t * L;
    if (i < n) gx[i] = sx[j * 33 + t];
  }
}

// Factor one system per thread in FP64 (Sec. 2.4), round the factors to FP32
// into the warp-per-system layout, and build each lane-chunk's 2x2 transfer
// maps from the rounded factors.
__global__ void k_factor32(DevPlan P, int n, int L, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ c, const double* __restrict__ d, const double* __restrict__ e,
                           const double* __restrict__ sigma, float* __restrict__ fac, float* __restrict__ phi) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nsys = P.shared ? 1 : P.batch;
  if (s >= nsys) return;
  const int64_t o = P.shared ? 0 : s * (int64_t)n;
  const double sg = sigma ? sigma[s] : 0.0;
  const int64_t plane = 32 * (int64_t)L;
  float* F = fac + s * 5 * plane;
  float* Ph = phi + s * 32 * 8;
  double gam2 = 0.0, del2 = 0.0, gam1 = 0.0, del1 = 0.0;
  bool failed = false;
  double f00 = 1, f01 = 0, f10 = 0, f11 = 1;  // forward chunk map accumulator
  double t00 = 1, t01 = 0, t10 = 0, t11 = 1;  // backward chunk map accumulator
  for (int i = 0; i < 32 * L; ++i) {
    float ainv = 1.f, bp = 0.f, ep = 0.f, ga = 0.f, de = 0.f;
    if (i < n && !failed) {
      double ar, br, cr, dr, er;
      if (sigma) {
        float w[5];
        d4_weights_f(i, n, w);
        ar = sg * w[0];
        br = sg * w[1];
        cr = 1.0 + sg * w[2];
        dr = sg * w[3];
        er = sg * w[4];
      } else {
        cr = c[o + i];
        ar = (i >= 2) ? a[o + i] : 0.0;
        br = (i >= 1) ? b[o + i] : 0.0;
        dr = (i + 1 < n) ? d[o + i] : 0.0;
        er = (i + 2 < n) ? e[o + i] : 0.0;
      }
      if (i < 2) ar = 0.0;
      if (i < 1) br = 0.0;
      if (i + 1 >= n) dr = 0.0;
      if (i + 2 >= n) er = 0.0;
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
        bp = (float)(beta / alpha);
        ep = (float)(ar / alpha);
        ga = (float)gamma;
        de = (float)delta;
        gam2 = gam1;
        del2 = del1;
        gam1 = gamma;
        del1 = delta;
      }
    }
    const int t = i / L, j = i - t * L;
    F[0 * plane + j * 32 + t] = ainv;
    F[1 * plane + j * 32 + t] = bp;
    F[2 * plane + j * 32 + t] = ep;
    F[3 * plane + j * 32 + t] = ga;
    F[4 * plane + j * 32 + t] = de;
    // forward row map M = [[0, 1], [-ep, -bp]] applied after the accumulated ones: acc <- M acc
    {
      const double n00 = f10, n01 = f11;
      const double n10 = -(double)ep * f00 - (double)bp * f10;
      const double n11 = -(double)ep * f01 - (double)bp * f11;
      f00 = n00; f01 = n01; f10 = n10; f11 = n11;
    }
    // backward row map B = [[-ga, -de], [1, 0]] applied before the accumulated ones: acc <- acc B
    {
      const double n00 = -t00 * (double)ga + t01, n01 = -t00 * (double)de;
      const double n10 = -t10 * (double)ga + t11, n11 = -t10 * (double)de;
      t00 = n00; t01 = n01; t10 = n10; t11 = n11;
    }
    if (j == L - 1) {
      float* q = Ph + t * 8;
      q[0] = (float)f00; q[1] = (float)f01; q[2] = (float)f10; q[3] = (float)f11;
      q[4] = (float)t00; q[5] = (float)t01; q[6] = (float)t10; q[7] = (float)t11;
      f00 = 1; f01 = 0; f10 = 0; f11 = 1;
      t00 = 1; t01 = 0; t10 = 0; t11 = 1;
    }
  }
}

template <int L>
cudaError_t launch_solve32r_L(int64_t batch, int n, int shared, const F32Factors& F, const double* sigma,
                              const double* f, double* x, int max_refine, int tol_log2, unsigned long long* info,
                              cudaStream_t st) {
  constexpr int kBytesPerWarp = 5 * 32 * L * 4 + L * 33 * 8;
  int warps = (int)((200 * 1024) / kBytesPerWarp);
  warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
  const size_t smem = (size_t)warps * kBytesPerWarp;
  static bool attr_set = false;  // once per process (the attribute is not a stream operation)
  if (!attr_set) {
    cudaError_t err = cudaFuncSetAttribute(k_solve32r<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set = true;
  }
  const int64_t grid = (batch + warps - 1) / warps;
  k_solve32r<L><<<(unsigned)grid, 32 * warps, smem, st>>>(batch, n, shared, F.fac, F.phi, sigma, f, x, max_refine,
                                                         tol_log2, info);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_factor32(const DevPlan& P, const double* a, const double* b, const double* c, const double* d,
                            const double* e, const double* sigma, F32Factors F, int n, cudaStream_t st) {
  const int64_t nsys = P.shared ? 1 : P.batch;
  const int block = 128;
  k_factor32<<<(unsigned)((nsys + block - 1) / block), block, 0, st>>>(P, n, F.L, a, b, c, d, e, sigma, F.fac, F.phi);
  return cudaGetLastError();
}

cudaError_t launch_solve32r(const DevPlan& P, F32Factors F, const double* sigma, int n, const double* f, double* x,
                            int max_refine, int residual_f64, int tol_log2, cudaStream_t st) {
  (void)residual_f64;
  switch (F.L) {
    case 2: return launch_solve32r_L<2>(P.batch, n, P.shared, F, sigma, f, x, max_refine, tol_log2, P.info, st);
    case 4: return launch_solve32r_L<4>(P.batch, n, P.shared, F, sigma, f, x, max_refine, tol_log2, P.info, st);
    case 8: return launch_solve32r_L<8>(P.batch, n, P.shared, F, sigma, f, x, max_refine, tol_log2, P.info, st);
    case 16: return launch_solve32r_L<16>(P.batch, n, P.shared, F, sigma, f, x, max_refine, tol_log2, P.info, st);
    case 32: return launch_solve32r_L<32>(P.batch, n, P.shared, F, sigma, f, x, max_refine, tol_log2, P.info, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pent
