// Float-float ("double-FP32") building blocks shared by the FP32 solve kernels:
// error-free transformations, the integer split of FP64 values into float
// pairs and their reassembly, the no-flux fourth-difference weights, 2x2 map
// helpers for the chunk scans, and the float-float residual of one row of
// A = I + sigma D4.  Device-only; every function is inlined into its caller
// (the one out-of-line slow path is static to each translation unit).
#pragma once

#include <cmath>
#include <cstdint>

namespace pent {
namespace ff {

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
// lo: the next 23 bits, rounded to nearest; together 47 bits, a relative error
// below 2^-48, unbiased so that it does not build up over many time steps),
// using integer operations only.  Values whose scaled magnitude is below
// 2^-126 are flushed to zero; the caller picks k so that the largest |v| of the
// system scales to just below 1.
__device__ __forceinline__ void split_scaled(double v, int k, float& hi, float& lo) {
  const unsigned long long U = (unsigned long long)__double_as_longlong(v);
  const unsigned top = (unsigned)(U >> 32), bot = (unsigned)U;
  const int E = (int)((top >> 20) & 0x7ffu);
  const int Es = E - k;
  const unsigned sign = top & 0x80000000u;
  const unsigned mant_hi = __funnelshift_l(bot, top, 3) & 0x7fffffu;  // mantissa bits 29..51
  const unsigned hib = sign | ((unsigned)(Es - 896) << 23) | mant_hi;
  // mantissa bits 6..28 (the 23 below hi's), rounded by bit 5; 2^23 still converts exactly below
  const unsigned rem = ((bot >> 6) & 0x7fffffu) + ((bot >> 5) & 1u);
  const float scale = __uint_as_float((unsigned)(Es - 942) << 23);  // 2^(Es - 1069)
  const unsigned lob = __float_as_uint(__fmul_rn(small_uint_to_float(rem), scale)) ^ sign;
  // branch-free: values that scale below FP32's normal range flush to zero
  const bool okh = (E != 0) && (Es >= 897), okl = okh && (Es >= 943);
  hi = okh ? __uint_as_float(hib) : 0.0f;
  lo = okl ? __uint_as_float(lob) : 0.0f;
}

// Rare path of ff_to_double_shift (h outside the range the fast path covers):
// exact conversions and one FP64 add, out of line.
static __device__ __noinline__ double ff_to_double_slow(float h, float l, int k) { return ldexp((double)h, k) + ldexp((double)l, k); }

// (h + l) * 2^k as a double for a normalised float-float pair (|l| <= ulp(h) / 2),
// without FP64 instructions: h's bits are moved into a double, and l, counted
// in units in the last place of that double (l * 2^(52 - e(h)), an integer
// below 2^29 in magnitude, rounded to nearest: an error of at most half a unit),
// is added to its 64-bit pattern.  Where h is a power of two and the sum is
// smaller, it falls in the binade below, whose units are half as large.  The
// sum cannot reach the binade above (|l| <= ulp(h) / 2).  The fast path needs
// 2^-74 <= |h| < 2^128 (so that l's scaling stays in the normal float range);
// the caller's scaling puts every nonzero |x| there unless it lies 75 binades
// below the largest.
__device__ __forceinline__ double ff_to_double_shift(float h, float l, int k) {
  const unsigned uh = __float_as_uint(h);
  const unsigned ah = uh & 0x7fffffffu;
  const int eh = (int)(ah >> 23);
  if (ah == 0u) return 0.0;  // then l == 0 too
  if (eh < 53 || eh == 255 || eh + 896 + k < 2 || eh + 896 + k > 2045) return ff_to_double_slow(h, l, k);
  // l in units of the double's last place, signed as the change of |h + l|
  const float units = __fmul_rn(l, __uint_as_float((unsigned)(306 - eh) << 23));  // l * 2^(179 - eh) = l * 2^(52 - e(h))
  int kk = __float2int_rn(units);
  kk = (uh & 0x80000000u) ? -kk : kk;
  if ((ah & 0x7fffffu) == 0u && kk < 0) kk *= 2;
  const unsigned long long bits = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                  (((unsigned long long)ah + ((unsigned long long)(896 + k) << 23)) << 29);
  return __longlong_as_double((long long)(bits + (unsigned long long)(long long)kk));
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

// ---------------------------------------------------------------- chunk maps and scans

// 2x2 matrices are float4 (x y / z w, row-major); states are (c0, c1).
__device__ __forceinline__ float4 mmul(const float4 a, const float4 b) {  // a * b
  return make_float4(fmaf(a.x, b.x, a.y * b.z), fmaf(a.x, b.y, a.y * b.w), fmaf(a.z, b.x, a.w * b.z),
                     fmaf(a.z, b.y, a.w * b.w));
}

__device__ __forceinline__ float mnorm(const float4 m) {
  return fmaxf(fmaxf(fabsf(m.x), fabsf(m.y)), fmaxf(fabsf(m.z), fabsf(m.w)));
}

// Value of lane - d (UP) or lane + d (down) of the warp.
template <bool UP>
__device__ __forceinline__ float shfl(float v, int d) {
  return UP ? __shfl_up_sync(0xffffffffu, v, d) : __shfl_down_sync(0xffffffffu, v, d);
}
template <bool UP>
__device__ __forceinline__ float4 shfl4(const float4 v, int d) {
  return make_float4(shfl<UP>(v.x, d), shfl<UP>(v.y, d), shfl<UP>(v.z, d), shfl<UP>(v.w, d));
}

// c <- m c + b.
__device__ __forceinline__ void apply(const float4 m, const float2 b, float& c0, float& c1) {
  const float n0 = fmaf(m.x, c0, fmaf(m.y, c1, b.x));
  const float n1 = fmaf(m.z, c0, fmaf(m.w, c1, b.y));
  c0 = n0;
  c1 = n1;
}


// r = f - (I + sigma D4) x for one row, in float-float (x = xh + xl, f = fh + fl,
// sigma = sgh + sgl), rounded to FP32, with the [1, -4, 6, -4, 1] stencil on
// the row's neighbours a, b, (c), d, e.  Rows next to a wall get their
// reflected (ghost) neighbours from the caller.
__device__ __forceinline__ float residual_row(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                              float dl, float eh, float el, float fhj, float flj, float sgh,
                                              float sgl) {
  float s1, e1, s2, e2, t, e3, p, e4, S, Er;
  two_sum(ah, eh, s1, e1);        // x_{i-2} + x_{i+2}
  two_sum(bh, dh, s2, e2);        // x_{i-1} + x_{i+1}
  two_sum(s1, -4.f * s2, t, e3);  // 4 s2 is exact
  two_prod(6.f, ch, p, e4);
  two_sum(t, p, S, Er);
  const float low = fmaf(6.f, cl, fmaf(-4.f, bl + dl, al + el));
  Er = Er + ((e1 - 4.f * e2) + (e3 + e4) + low);
  float yh, yl;
  fast_two_sum(S, Er, yh, yl);
  float Pp, Pe;  // sigma * y
  two_prod(sgh, yh, Pp, Pe);
  Pe = fmaf(sgh, yl, fmaf(sgl, yh, Pe));
  float a1, a2, b1, b2;
  two_sum(fhj, -ch, a1, a2);
  two_sum(a1, -Pp, b1, b2);
  const float lo2 = ((a2 + b2) + (flj - cl)) - Pe;
  return b1 + lo2;
}

// Index of the row whose value the cell-centred no-flux walls reflect into
// position g of an n-row system (-1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2, and
// repeatedly for systems shorter than the stencil).
__device__ __forceinline__ int reflect_row(int g, int n) {
  while (g < 0 || g >= n) g = (g < 0) ? (-1 - g) : (2 * n - 1 - g);
  return g;
}

// Replace the ghost entries of a neighbour window w[0 .. L+3] (rows tg L - 2 ..
// tg L + L + 1 of the system) by the rows the walls reflect them to.  Only the
// first chunk of a system and the chunks whose window reaches row n have ghosts, and
// for n >= 4 each ghost is a copy of a real row two or fewer positions away
// (w[k] for row -1 is row 0, for row n it is row n - 1, ...).  Systems with
// n < 4 lie in one chunk and take the general reflection.
template <int L>
__device__ __forceinline__ void fill_ghosts(float (&w)[L + 4], int tg, int n) {
  const int m = n - tg * L;  // row n sits at window position m + 2
  if (n < 4) {
    if (tg == 0) {
      float src[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) src[k] = w[2 + k];
#pragma unroll
      for (int q = 0; q < L + 4; ++q) {
        const int g = reflect_row(q - 2, n);  // 0 <= g < n <= 3
        w[q] = (g == 0) ? src[0] : ((g == 1) ? src[1] : src[2]);
      }
    }
    return;
  }
  if (tg == 0) {  // rows -2, -1 reflect to 1, 0
    w[0] = w[3];
    w[1] = w[2];
  }
  if (m >= 1 && m <= L + 1) {  // rows n, n + 1 (inside the window) reflect to n - 1, n - 2
#pragma unroll
    for (int q = 3; q < L + 4; ++q) {
      if (q - 2 == m)
        w[q] = w[q - 1];
      else if (q - 2 == m + 1)
        w[q] = w[q - 3];
    }
  }
}

// The neighbouring rows of this thread's chunk: the last two rows of the

}  // namespace ff
}  // namespace pent
