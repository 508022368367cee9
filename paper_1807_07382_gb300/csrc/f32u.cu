// FP32 substitution with one refinement step for hyperdiffusion systems whose
// factors are constant away from the walls.
//
// The factorisation of A = I + sigma D4 (Sec. 2.4, factorisation steps) is a
// recurrence whose coefficients are the same on every interior row, and it
// settles: once the FP32 values of 1/alpha_i and beta_i stop changing they stay
// at one fixed pair up to row n - 3 (for sigma <= 10 from row 21 on at the
// latest; the two rows at the right wall differ again).  So a system is three
// stretches: the head rows 0 .. K-1 with their own factors, the interior rows
// K .. n-3 where both substitutions (Sec. 2.4: L g = f, then R x = g) are
// recurrences with the same two constants, and the two tail rows.
//
// One CTA of P = 32 W threads owns one system, thread t holding rows
// t L .. t L + L - 1 in registers, as in csrc/f32r.cu.  A thread whose chunk
// lies in the interior does not load factors at all: it uses the pair of
// constants, and every interior chunk acts on the two carried values with the
// same affine map whose linear part M is one 2x2 matrix per system.  The scan
// that joins the chunks therefore needs only powers of M -- M^(2^l) for the
// Kogge-Stone levels, M^k for a lane k positions into its warp, M^32 across
// warps -- which the factorisation stores once per system (k_uplan32), instead
// of a per-lane plan built in every launch.  The few chunks at the walls run
// their exact recurrence one after another ("chains"), the first from the
// system's boundary and the last from the state the scan hands them; the head
// chain's final state enters the interior scan as the affine part of the last
// head chunk, so every interior lane's entering state comes out of the same
// uniform scan.
//
// The refinement is that of csrc/f32r.cu: the residual f - A x in float-float
// (error-free transformations) with the walls' reflected neighbours, an FP32
// solve for the correction, and x = x + dx in float-float.  Across the steps of
// one CUDA-graph time loop the field can stay a float pair per row (scaled by a
// per-system power of two kept in `kscale`): only the first step splits the
// FP64 input and only the last reassembles FP64, so the steps in between carry
// no conversion work.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "ff.cuh"
#include "internal.cuh"

namespace pent {
namespace {

using namespace ff;

constexpr float kUTol = 9.3132257e-10f;  // 2^-30: coupling dropped from the scans (as in csrc/f32r.cu)
constexpr unsigned kFull = 0xffffffffu;

// Per-system record (float4 units): the constants, K and the scan levels, then
// for the forward (1 ..) and the back (39 ..) chunk map: M^(2^l), l = 0..5, and
// M^k, k = 0..31.
constexpr int kUFwd2 = 1, kUFwdK = 7, kUBwd2 = 39, kUBwdK = 45;
static_assert(kUBwdK + 32 == kURecFloat4, "record size");

// Factor slots in shared memory for the chains: head lanes 0..31 and up to four tail lanes
// (2 L + 4 floats each: 1/alpha and beta of the lane's rows, beta of the next row, padding to
// whole float4).  Chain lanes beyond these read their factors from global memory.
constexpr int kHeadSlots = 32, kTailSlots = 4;

// Dynamic shared memory of one CTA of W warps and L rows a thread: the system's record,
// the residual's edge rows, the right-hand side as float pairs (kept here between the
// first solve and the residual, to spare registers), four rotating sets of warp totals,
// the chains' hand-over slots, a reduction slot per warp, the chains' factor slots.
// Every float4 array comes first (16-byte aligned), then the float2 and int arrays.
__host__ __device__ constexpr int uslot_f4(int L) { return (2 * L + 4) / 4; }  // float4 per factor slot
__host__ __device__ inline size_t usmem_bytes(int W, int L) {
  const size_t P = 32 * (size_t)W;
  return sizeof(float4) * (kURecFloat4 + P + 2 * (size_t)(L / 4) * P + (kHeadSlots + kTailSlots) * (size_t)uslot_f4(L)) +
         sizeof(float2) * (4 * (size_t)W + 8) + sizeof(int) * (size_t)W;
}

// Value of lane - d (UP) or lane + d (down) of the warp.
template <bool UP>
__device__ __forceinline__ float ushfl(float v, int d) {
  return UP ? __shfl_up_sync(kFull, v, d) : __shfl_down_sync(kFull, v, d);
}

struct UCtx {
  int t, lane, warp;
  int n, H, T0, T1;  // head lanes [0, H), interior [H, T0), tail [T0, T1], padding after T1
  float ia, bi, sg;  // interior 1/alpha and beta, sigma (FP32 high part)
  int nlev_f, nlev_b;
  bool wsmall_f, wsmall_b;  // M^32 below the tolerance: only the previous warp carries
  const float4* rec;  // the system's record (shared memory)
  float4* fsl;        // chain factor slots (shared memory)
  const float4* gq;   // the system's factor block (k_factor32 layout)
  int PT;            // threads of the factor block
  int tg0;           // factor-block thread of this CTA's lane 0 (a window's first row / L)
  bool lw, rw;       // the CTA's first / last row is the system's wall (else a window's cut)
  int phase;
  float2* tot;   // [4][W] warp totals of one scan (rotating)
  float2* hand;  // [8] chain hand-over slots across warps
};

// This thread's FP32 factors (1/alpha, beta of its L rows and beta of the next row).
template <int L>
__device__ __forceinline__ void load_own(const UCtx& cx, float (&A)[L], float (&B)[L], float& bnext) {
#pragma unroll
  for (int jq = 0; jq < L / 4; ++jq) {
    const float4 qa = __ldg(cx.gq + (int64_t)(jq * 2 + 0) * cx.PT + cx.tg0 + cx.t),
                 qb = __ldg(cx.gq + (int64_t)(jq * 2 + 1) * cx.PT + cx.tg0 + cx.t);
    A[4 * jq] = qa.x; A[4 * jq + 1] = qa.y; A[4 * jq + 2] = qa.z; A[4 * jq + 3] = qa.w;
    B[4 * jq] = qb.x; B[4 * jq + 1] = qb.y; B[4 * jq + 2] = qb.z; B[4 * jq + 3] = qb.w;
  }
  const int tn = cx.tg0 + cx.t + 1;
  bnext = (tn < cx.PT) ? __ldg(reinterpret_cast<const float*>(cx.gq + (int64_t)cx.PT + tn)) : 0.f;
}

// Shared-memory factor slot of a chain lane, or -1 (then the factors come from global memory).
__device__ __forceinline__ int fslot(const UCtx& cx, int t) {
  if (t < cx.H && t < kHeadSlots) return t;
  if (t >= cx.T0 && t <= cx.T1 && t - cx.T0 < kTailSlots) return kHeadSlots + (t - cx.T0);
  return -1;
}

// The exact recurrence of this thread's chunk from the entering state (s0, s1):
// forward g_i = (1/alpha_i)(v_i - beta_i g_{i-1} - sigma g_{i-2}), state
// (g_{i-2}, g_{i-1}); back x_i = g_i - (1/alpha_i)(beta_{i+1} x_{i+1} + sigma
// x_{i+2}), state (x_{i+1}, x_{i+2}).  Leaves the state after the chunk.
template <int L, bool FWD>
__device__ __forceinline__ void pass_own(float (&v)[L], const UCtx& cx, float& s0, float& s1) {
  float A[L], B[L], bn;
  const int k = fslot(cx, cx.t);
  if (k >= 0) {
    const float4* q = cx.fsl + k * uslot_f4(L);
#pragma unroll
    for (int jq = 0; jq < L / 4; ++jq) {
      const float4 a = q[jq], b = q[L / 4 + jq];
      A[4 * jq] = a.x; A[4 * jq + 1] = a.y; A[4 * jq + 2] = a.z; A[4 * jq + 3] = a.w;
      B[4 * jq] = b.x; B[4 * jq + 1] = b.y; B[4 * jq + 2] = b.z; B[4 * jq + 3] = b.w;
    }
    bn = q[L / 2].x;
  } else {
    load_own<L>(cx, A, B, bn);
  }
  const float sg = cx.sg;
  if (FWD) {
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const float g = A[j] * fmaf(-B[j], s1, fmaf(-sg, s0, v[j]));
      v[j] = g;
      s0 = s1;
      s1 = g;
    }
  } else {
#pragma unroll
    for (int j = L - 1; j >= 0; --j) {
      const float b = (j + 1 < L) ? B[j + 1] : bn;
      const float xv = fmaf(-A[j], fmaf(b, s0, sg * s1), v[j]);
      v[j] = xv;
      s1 = s0;
      s0 = xv;
    }
  }
}

// Lanes [a, b] in sweep order (FWD: a .. b, else b .. a), one after another,
// each running its exact recurrence from the state the previous one left; the
// first enters with the (s0, s1) it holds.  Every lane ends with the chain's
// final state in (s0, s1) if its warp ran the last segment.  a, b are uniform
// over the CTA; a chain that crosses warps hands the state over through
// shared memory with one barrier per crossing.
template <int L, bool FWD>
__device__ __forceinline__ void chain(float (&v)[L], int a, int b, UCtx& cx, float& s0, float& s1, float2* slot) {
  if (a > b) return;
  const int wa = a >> 5, wb = b >> 5;
  for (int k = 0; k <= wb - wa; ++k) {
    const int w = FWD ? wa + k : wb - k;
    if (k > 0) __syncthreads();
    if (cx.warp == w) {
      if (k > 0) {
        const float2 q = *slot;
        s0 = q.x;
        s1 = q.y;
      }
      const int lo = max(a, 32 * w), hi = min(b, 32 * w + 31);
      for (int q = 0; q <= hi - lo; ++q) {
        const int j = FWD ? lo + q : hi - q;
        if (cx.t == j) pass_own<L, FWD>(v, cx, s0, s1);
        s0 = __shfl_sync(kFull, s0, j & 31);
        s1 = __shfl_sync(kFull, s1, j & 31);
      }
      if (k < wb - wa && cx.lane == 0) *slot = make_float2(s0, s1);
    }
  }
}

// Entering state of this lane's chunk for a sweep through the CTA's chunks in
// order (FWD: increasing lanes, else decreasing) when every chunk acts as
// (c0, c1) -> M (c0, c1) + u: Kogge-Stone over the warp with the stored powers
// M^(2^l), the warps' totals through shared memory, and the warp's entering
// state carried in by M^k, k this lane's position in its warp.
template <bool FWD>
__device__ __forceinline__ void scan_u(float u0, float u1, UCtx& cx, int W, float& e0, float& e1) {
  const float4* P2 = cx.rec + (FWD ? kUFwd2 : kUBwd2);
  const float4* PK = cx.rec + (FWD ? kUFwdK : kUBwdK);
  const int nlev = FWD ? cx.nlev_f : cx.nlev_b;
  const int lane = cx.lane;
#pragma unroll 1
  for (int l = 0; l < nlev; ++l) {
    const int d = 1 << l;
    const float o0 = ushfl<FWD>(u0, d), o1 = ushfl<FWD>(u1, d);
    if (FWD ? (lane >= d) : (lane + d < 32)) {
      const float4 m = P2[l];
      u0 = fmaf(m.x, o0, fmaf(m.y, o1, u0));
      u1 = fmaf(m.z, o0, fmaf(m.w, o1, u1));
    }
  }
  const bool first = FWD ? (lane == 0) : (lane == 31);
  float p0 = ushfl<FWD>(u0, 1), p1 = ushfl<FWD>(u1, 1);  // inclusive result of the previous chunk
  if (first) p0 = p1 = 0.f;
  float c0 = 0.f, c1 = 0.f;  // state entering this warp
  if (W > 1) {
    float2* tt = cx.tot + (cx.phase++ & 3) * W;
    if (FWD ? (lane == 31) : (lane == 0)) tt[cx.warp] = make_float2(u0, u1);
    __syncthreads();
    const bool small = FWD ? cx.wsmall_f : cx.wsmall_b;
    const int prev = FWD ? cx.warp - 1 : cx.warp + 1;
    if (small) {
      if (prev >= 0 && prev < W) {
        const float2 q = tt[prev];
        c0 = q.x;
        c1 = q.y;
      }
    } else {
      const float4 mw = P2[5];  // M^32
      const int cnt = FWD ? cx.warp : W - 1 - cx.warp;
      for (int k = 0; k < cnt; ++k) {
        const float2 q = tt[FWD ? k : W - 1 - k];
        const float n0 = fmaf(mw.x, c0, fmaf(mw.y, c1, q.x));
        const float n1 = fmaf(mw.z, c0, fmaf(mw.w, c1, q.y));
        c0 = n0;
        c1 = n1;
      }
    }
  }
  const float4 mk = PK[FWD ? lane : 31 - lane];
  e0 = fmaf(mk.x, c0, fmaf(mk.y, c1, p0));
  e1 = fmaf(mk.z, c0, fmaf(mk.w, c1, p1));
}

// In place v <- A^{-1} v in FP32 (forward, then back substitution).
template <int L>
__device__ __forceinline__ void solve_u(float (&v)[L], UCtx& cx, int W) {
  const int t = cx.t;
  const bool interior = t >= cx.H && t < cx.T0;
  const float ia = cx.ia, bi = cx.bi, sg = cx.sg;
  // ---- forward ----
  float u0 = 0.f, u1 = 0.f;
  if (interior) {
    float p2 = 0.f, p1 = 0.f;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const float g = ia * fmaf(-bi, p1, fmaf(-sg, p2, v[j]));
      p2 = p1;
      p1 = g;
    }
    u0 = p2;
    u1 = p1;
  }
  if (cx.H > 0) {  // head chunks from the left wall; the last one's state enters the scan
    float s0 = 0.f, s1 = 0.f;
    chain<L, true>(v, 0, cx.H - 1, cx, s0, s1, cx.hand + 0);
    if (t == cx.H - 1) {
      u0 = s0;
      u1 = s1;
    }
  }
  float e0, e1;
  scan_u<true>(u0, u1, cx, W, e0, e1);
  if (interior) {
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const float g = ia * fmaf(-bi, e1, fmaf(-sg, e0, v[j]));
      v[j] = g;
      e0 = e1;
      e1 = g;
    }
  }
  chain<L, true>(v, cx.T0, cx.T1, cx, e0, e1, cx.hand + 1);  // tail chunks from the scan's state
  if (t > cx.T1) {
#pragma unroll
    for (int j = 0; j < L; ++j) v[j] = 0.f;
  }
  // ---- back ----
  u0 = u1 = 0.f;
  {
    float s0 = 0.f, s1 = 0.f;  // the right wall: x_n = x_{n+1} = 0
    chain<L, false>(v, cx.T0, cx.T1, cx, s0, s1, cx.hand + 2);
    if (t == cx.T0 && cx.T0 <= cx.T1) {
      u0 = v[0];
      u1 = v[1];
    }
  }
  if (interior) {
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int j = L - 1; j >= 0; --j) {
      const float xv = fmaf(-ia, fmaf(bi, s1, sg * s2), v[j]);
      s2 = s1;
      s1 = xv;
    }
    u0 = s1;
    u1 = s2;
  }
  scan_u<false>(u0, u1, cx, W, e0, e1);
  if (interior) {
#pragma unroll
    for (int j = L - 1; j >= 0; --j) {
      const float xv = fmaf(-ia, fmaf(bi, e0, sg * e1), v[j]);
      v[j] = xv;
      e1 = e0;
      e0 = xv;
    }
  }
  if (cx.H > 0) {  // head chunks from the state of lane H (or the right wall)
    const int hb = cx.H - 1;
    float s0 = 0.f, s1 = 0.f;
    if (cx.H <= cx.T1) {
      if ((cx.H & 31) != 0) {  // lane H is in the same warp
        s0 = __shfl_down_sync(kFull, v[0], 1);
        s1 = __shfl_down_sync(kFull, v[1], 1);
      } else {
        if (t == cx.H) cx.hand[4] = make_float2(v[0], v[1]);
        __syncthreads();
        const float2 q = cx.hand[4];
        s0 = q.x;
        s1 = q.y;
      }
    }
    chain<L, false>(v, 0, hb, cx, s0, s1, cx.hand + 3);
  }
}

// Replace the ghost entries of the neighbour window w[0 .. L+3] (rows tg L - 2 ..
// tg L + L + 1 of a system of n >= 4 rows) by the rows the cell-centred walls
// reflect them to: rows -2, -1 are rows 1, 0; rows n, n+1 are rows n-1, n-2.
// lw = false: row 0 is not the wall (nothing reflects there); n may lie beyond
// every row of the window (no right wall).  Written as selects on fixed
// positions, so the window stays in registers.
template <int L>
__device__ __forceinline__ void ghosts_u(float (&w)[L + 4], int tg, int n, bool lw) {
  if (lw && tg == 0) {
    w[0] = w[3];
    w[1] = w[2];
  }
  const int m = n - tg * L;  // row n sits at window position m + 2
#pragma unroll
  for (int q = 3; q < L + 4; ++q) w[q] = (q - 2 == m) ? w[q - 1] : ((q - 3 == m) ? w[q - 3] : w[q]);
}

// Row g of a system of n <= 3 rows held in one thread's x[0 .. 2].
template <int L>
__device__ __forceinline__ float pick3(const float (&x)[L], int g) {
  return g == 0 ? x[0] : (g == 1 ? x[1] : x[2]);
}

// Float-float residual r = f - (I + sigma D4) xh of this thread's rows (xh in
// FP32: the first refinement step), with the rows of the neighbouring threads
// exchanged through shared memory and the walls' reflected ghosts; beyond a
// window's cut the rows count as zero (the window's own truncated system).
template <int L>
__device__ __forceinline__ void residual_u(const float4* fsm, const float (&xh)[L], float (&r)[L], float sgh,
                                           float sgl, const UCtx& cx, float4* edge, int P) {
  const int t = cx.t, n = cx.n;
  float fh[L], fl[L];
#pragma unroll
  for (int jq = 0; jq < L / 4; ++jq) {
    const float4 a = fsm[jq * P + t], b = fsm[(L / 4 + jq) * P + t];
    fh[4 * jq] = a.x; fh[4 * jq + 1] = a.y; fh[4 * jq + 2] = a.z; fh[4 * jq + 3] = a.w;
    fl[4 * jq] = b.x; fl[4 * jq + 1] = b.y; fl[4 * jq + 2] = b.z; fl[4 * jq + 3] = b.w;
  }
  edge[t] = make_float4(xh[0], xh[1], xh[L - 2], xh[L - 1]);
  __syncthreads();
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 prv = t > 0 ? edge[t - 1] : zero;
  const float4 nxt = t + 1 < P ? edge[t + 1] : zero;
  float wh[L + 4];  // rows t L - 2 .. t L + L + 1
  wh[0] = prv.z;
  wh[1] = prv.w;
  wh[L + 2] = nxt.x;
  wh[L + 3] = nxt.y;
#pragma unroll
  for (int j = 0; j < L; ++j) wh[j + 2] = xh[j];
  if (n >= 4) {
    ghosts_u<L>(wh, t, cx.rw ? n : (1 << 29), cx.lw);
  } else {  // one thread holds the whole system: every stencil column reflects into rows 0 .. n-1
#pragma unroll
    for (int q = 0; q < L + 4; ++q) wh[q] = pick3<L>(xh, reflect_row(q - 2, n));
  }
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float res = residual_row(wh[j], 0.f, wh[j + 1], 0.f, wh[j + 2], 0.f, wh[j + 3], 0.f, wh[j + 4], 0.f, fh[j],
                                   fl[j], sgh, sgl);
    r[j] = (t * L + j < n) ? res : 0.f;
  }
}

// Biased FP32 exponent of |h| (0 for zero).
__device__ __forceinline__ int fexp(float h) { return (int)((__float_as_uint(h) >> 23) & 0xffu); }

// IN / OUT: 0 = FP64 values, 1 = float pairs (h, l) per row scaled by 2^-kscale[s].
// REF: refinement steps (0 or 1).
// Warps per SM the register allocation must allow: 40 (ten CTAs of four warps, 51
// registers a thread; on GB300 65,536 x 1024 with one refinement step 0.558 ms a graph
// step, against 0.584 at 32 warps, where no register spills).
#ifndef PENT_U_WARPS_PER_SM
#define PENT_U_WARPS_PER_SM 40
#endif

// Warps per SM for the windows of long systems (FP64 in and out): 36 (56 registers a thread; on
// GB300 the uneven batch with 4-warp windows takes 0.686 ms a step against 0.695 at 32 warps, no
// spills, and 0.707 at 40).
#ifndef PENT_U_WIN_WARPS_PER_SM
#define PENT_U_WIN_WARPS_PER_SM 36
#endif

// CTAs per SM the launch bound asks for: PENT_U_WARPS_PER_SM (windows: PENT_U_WIN_WARPS_PER_SM)
// warps, or for the runtime-width kernel two CTAs of up to 16 warps (64 registers a thread).
constexpr int u_min_blocks(int WT, int WIN) {
  return WT > 0 ? (WIN ? PENT_U_WIN_WARPS_PER_SM : PENT_U_WARPS_PER_SM) / WT : 2;
}

// WIN = 1: the CTA solves window win[b] (b < nwin) = (system, first row w0, rows m | overlap
// rows O << 16) of a long system: rows w0 .. w0 + m - 1 as one system of m rows whose cuts (a
// first row other than 0, a last one other than n - 1) enter and leave with zero states,
// writing out only the rows at least O from a cut.  halo: the overlap rows of every window
// copied out before an in-place solve ([window][left, right][omax]), or nullptr (read from f).
struct UWinArgs {
  const int4* win;
  int64_t nwin;
  const int32_t* fshape;  // [nfac] threads | L << 16 of each factor block
  const double* halo;
  int omax;
};

// One system (or window) `item` solved by the CTA.
template <int L, int WT, int REF, int IN, int OUT, int WIN>
__device__ __forceinline__ void u_item(unsigned item, const F32Tables& T, const float4* __restrict__ urec,
                                       int32_t* __restrict__ kscale, const int32_t* __restrict__ sys, int shared,
                                       const double* f, double* x, int vec_io, int Wrt, const UWinArgs& wa) {
  static_assert(L % 4 == 0, "rows per thread must be a multiple of 4");
  static_assert(!WIN || (IN == 0 && OUT == 0), "windows read and write FP64");
  const int W = WT > 0 ? WT : Wrt, P = 32 * W;  // WT = 0: the warp count is a launch parameter
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* rec_sm = reinterpret_cast<float4*>(smem_raw);        // [kURecFloat4]
  float4* edge = rec_sm + kURecFloat4;                         // [P]
  float4* fsm = edge + P;                                      // [2 L / 4][P]: f high parts, then low parts
  float4* fsl = fsm + 2 * (L / 4) * P;                         // [kHeadSlots + kTailSlots][uslot_f4(L)]
  float2* tot = reinterpret_cast<float2*>(fsl + (kHeadSlots + kTailSlots) * uslot_f4(L));  // [4][W]
  float2* hand = tot + 4 * W;                                  // [8]
  int* redi = reinterpret_cast<int*>(hand + 8);                // [W]
  const int t = threadIdx.x;
  UCtx cx;
  cx.t = t;
  cx.lane = t & 31;
  cx.warp = t >> 5;
  cx.phase = 0;
  cx.tot = tot;
  cx.hand = hand;
  int64_t s;
  int n, w0 = 0, O = 0;  // rows of the CTA's system (or window), its first row, its overlap
  cx.tg0 = 0;
  cx.lw = cx.rw = true;
  if (WIN) {
    const int4 d = wa.win[item];
    s = d.x;
    w0 = d.y;
    n = d.z & 0xffff;
    O = d.z >> 16;
    cx.lw = w0 == 0;
    cx.rw = w0 + n == T.n[s];
    cx.tg0 = w0 / L;
  } else {
    s = sys[item];
    n = T.n[s];
  }
  const int64_t ms = shared ? 0 : s;
  cx.n = n;
  const float4* grec = urec + ms * kURecFloat4;
  for (int k = t; k < kURecFloat4; k += P) rec_sm[k] = __ldg(grec + k);
  cx.rec = rec_sm;
  cx.fsl = fsl;
  const float4 hd = __ldg(grec);
  cx.ia = hd.x;
  cx.bi = hd.y;
  const int K = __float_as_int(hd.z), flags = __float_as_int(hd.w);
  cx.nlev_f = flags & 0xff;
  cx.nlev_b = (flags >> 8) & 0xff;
  cx.wsmall_f = (flags >> 16) & 1;
  cx.wsmall_b = (flags >> 17) & 1;
  const float2 sgp = __ldg(T.sig2 + ms);
  cx.sg = sgp.x;
  cx.gq = reinterpret_cast<const float4*>(T.fac) + T.foff[ms];
  cx.PT = WIN ? (wa.fshape[ms] & 0xffff) : P;
  cx.T1 = (n - 1) / L;
  cx.H = cx.lw ? min((K + L - 1) / L, cx.T1 + 1) : 0;             // a cut: no head chain
  cx.T0 = cx.rw ? max(n >= 3 ? (n - 3) / L : 0, cx.H) : cx.T1 + 1;  // a cut: no tail chain
  const int i0 = t * L;
  {  // the chain lanes' factors, loaded once for all four sweeps
    const int k = fslot(cx, t);
    if (k >= 0) {
      float A[L], B[L], bn;
      load_own<L>(cx, A, B, bn);
      float4* q = fsl + k * uslot_f4(L);
#pragma unroll
      for (int jq = 0; jq < L / 4; ++jq) {
        q[jq] = make_float4(A[4 * jq], A[4 * jq + 1], A[4 * jq + 2], A[4 * jq + 3]);
        q[L / 4 + jq] = make_float4(B[4 * jq], B[4 * jq + 1], B[4 * jq + 2], B[4 * jq + 3]);
      }
      q[L / 2] = make_float4(bn, 0.f, 0.f, 0.f);
    }
  }
  __syncthreads();  // record and slots visible to the CTA

  // ---- right-hand side as a float pair per row ----
  float fh[L], fl[L];
  int kshift;
  bool store_k = false;
  if (IN == 0) {
    const double* src = f + T.off[s] + w0 + i0;  // this thread's first row
    if (WIN && wa.halo) {  // overlap rows (whole threads: O and the cuts are multiples of L)
      const bool lh = !cx.lw && i0 < O, rh = !cx.rw && i0 >= n - O;
      const double* hb = wa.halo + (int64_t)item * 2 * wa.omax;
      if (lh) src = hb + i0;
      if (rh) src = hb + wa.omax + (i0 - (n - O));
    }
    double fv[L];
    if (vec_io && i0 + L <= n) {
#pragma unroll
      for (int j = 0; j < L; j += 2) {
        const double2 q = *reinterpret_cast<const double2*>(src + j);
        fv[j] = q.x;
        fv[j + 1] = q.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < L; ++j) fv[j] = (i0 + j < n) ? src[j] : 0.0;
    }
    int emax = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const unsigned top = (unsigned)((unsigned long long)__double_as_longlong(fv[j]) >> 32);
      emax = max(emax, (int)((top >> 20) & 0x7ffu));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) emax = max(emax, __shfl_xor_sync(kFull, emax, d));
    if (W > 1) {
      if (cx.lane == 0) redi[cx.warp] = emax;
      __syncthreads();
      for (int w = 0; w < W; ++w) emax = max(emax, redi[w]);
    }
    kshift = emax - 1022;  // the largest |f| scales into [1/2, 1)
#pragma unroll
    for (int j = 0; j < L; ++j) split_scaled(fv[j], kshift, fh[j], fl[j]);
    store_k = true;
  } else {
    const float* fs = reinterpret_cast<const float*>(f + T.off[s]);
    if (vec_io && i0 + L <= n) {
#pragma unroll
      for (int j = 0; j < L; j += 2) {
        const float4 q = *reinterpret_cast<const float4*>(fs + 2 * (i0 + j));
        fh[j] = q.x;
        fl[j] = q.y;
        fh[j + 1] = q.z;
        fl[j + 1] = q.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const bool in = i0 + j < n;
        fh[j] = in ? fs[2 * (i0 + j)] : 0.f;
        fl[j] = in ? fs[2 * (i0 + j) + 1] : 0.f;
      }
    }
    kshift = kscale[s];
    // a field that has decayed far below its scale is rescaled (the low parts would leave FP32's range)
    int em = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) em = max(em, fexp(fh[j]));
    if (__syncthreads_and(em < 126 - 60)) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) em = max(em, __shfl_xor_sync(kFull, em, d));
      if (W > 1) {
        if (cx.lane == 0) redi[cx.warp] = em;
        __syncthreads();
        for (int w = 0; w < W; ++w) em = max(em, redi[w]);
      }
      if (em > 0) {
        const int d = 126 - em;  // the largest |h| scales into [1/2, 1)
        const float sc = __uint_as_float((unsigned)(127 + d) << 23);
#pragma unroll
        for (int j = 0; j < L; ++j) {
          fh[j] *= sc;
          fl[j] *= sc;
        }
        kshift -= d;
        store_k = true;
      }
    }
  }

  // ---- FP32 solve, then (REF = 1) the float-float residual, its FP32 solve and the
  // correction; one solve call site keeps the kernel's code compact (instruction cache) ----
  float v[L], xh[L], xl[L];
#pragma unroll
  for (int j = 0; j < L; ++j) v[j] = fh[j];
  if (REF > 0) {  // this thread's f for the residual (its own slots: no barrier needed)
#pragma unroll
    for (int jq = 0; jq < L / 4; ++jq) {
      fsm[jq * P + t] = make_float4(fh[4 * jq], fh[4 * jq + 1], fh[4 * jq + 2], fh[4 * jq + 3]);
      fsm[(L / 4 + jq) * P + t] = make_float4(fl[4 * jq], fl[4 * jq + 1], fl[4 * jq + 2], fl[4 * jq + 3]);
    }
  }
#pragma unroll 1
  for (int it = 0; it <= REF; ++it) {
    if (it > 0) residual_u<L>(fsm, xh, v, sgp.x, sgp.y, cx, edge, P);
    solve_u<L>(v, cx, W);
    if (it == 0) {
#pragma unroll
      for (int j = 0; j < L; ++j) xh[j] = v[j];
    }
  }
  if (REF > 0) {  // x = x0 + dx in float-float
#pragma unroll
    for (int j = 0; j < L; ++j) {
      float sh, se;
      two_sum(xh[j], v[j], sh, se);
      fast_two_sum(sh, se, xh[j], xl[j]);
    }
    if (item == 0 && t == 0) atomicMax(T.info + 1, (unsigned long long)REF);
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j) xl[j] = 0.f;
  }

  // ---- store ----
  if (OUT == 0) {
    double* xs = x + T.off[s] + w0;
    const int o0 = cx.lw ? 0 : O, o1 = cx.rw ? n : n - O;  // rows written out (a window: its own rows)
    double xv[L];
#pragma unroll
    for (int j = 0; j < L; ++j) xv[j] = ff_to_double_shift(xh[j], xl[j], kshift);
    if (vec_io && i0 >= o0 && i0 + L <= o1) {
#pragma unroll
      for (int j = 0; j < L; j += 2) *reinterpret_cast<double2*>(xs + i0 + j) = make_double2(xv[j], xv[j + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < L; ++j)
        if (i0 + j >= o0 && i0 + j < o1) xs[i0 + j] = xv[j];
    }
  } else {
    float* xs = reinterpret_cast<float*>(x + T.off[s]);
    if (vec_io && i0 + L <= n) {
#pragma unroll
      for (int j = 0; j < L; j += 2)
        *reinterpret_cast<float4*>(xs + 2 * (i0 + j)) = make_float4(xh[j], xl[j], xh[j + 1], xl[j + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < L; ++j)
        if (i0 + j < n) *reinterpret_cast<float2*>(xs + 2 * (i0 + j)) = make_float2(xh[j], xl[j]);
    }
    if (store_k && t == 0) kscale[s] = kshift;
  }
}

// A CTA per system (WIN = 0) or window (WIN = 1); WIN = 2 is the persistent form of the windows,
// a grid of resident CTAs that take the windows in turn.
template <int L, int WT, int REF, int IN, int OUT, int WIN>
__global__ void __launch_bounds__(WT > 0 ? 32 * WT : 512, u_min_blocks(WT, WIN))
    k_solve32u(F32Tables T, const float4* __restrict__ urec, int32_t* __restrict__ kscale,
               const int32_t* __restrict__ sys, int shared, const double* f, double* x, int vec_io, int Wrt,
               UWinArgs wa) {
  if (WIN == 2) {
    for (unsigned item = blockIdx.x; item < wa.nwin; item += gridDim.x) {
      u_item<L, WT, REF, IN, OUT, WIN>(item, T, urec, kscale, sys, shared, f, x, vec_io, Wrt, wa);
      __syncthreads();  // the next window reuses the shared memory
    }
  } else {
    u_item<L, WT, REF, IN, OUT, WIN>(blockIdx.x, T, urec, kscale, sys, shared, f, x, vec_io, Wrt, wa);
  }
}

// ---------------------------------------------------------------- per-system record (once per factorisation)

// 2x2 products in FP64 (rounded to FP32 when stored).
struct M2 {
  double a, b, c, d;
};
__device__ __forceinline__ M2 mul2(const M2& p, const M2& q) {
  return M2{p.a * q.a + p.b * q.c, p.a * q.b + p.b * q.d, p.c * q.a + p.d * q.c, p.c * q.b + p.d * q.d};
}
__device__ __forceinline__ float4 to_f4(const M2& m) {
  return make_float4((float)m.a, (float)m.b, (float)m.c, (float)m.d);
}
__device__ __forceinline__ double norm2(const M2& m) {
  return fmax(fmax(fabs(m.a), fabs(m.b)), fmax(fabs(m.c), fabs(m.d)));
}

// One warp per factor block: K (the first row of the run of equal FP32 factor
// pairs that ends at row n - 3), the interior pair, and the powers of the
// interior chunk maps of L rows -- forward on (g_{i-2}, g_{i-1}), back on
// (x_{i+1}, x_{i+2}), the recurrences of pass_own with constant factors.
// uwin (if set): (K, O) per factor block, O the overlap rows a window of the system needs: the
// fewest whole chunks k L with |M^k| <= 2^-56 for both chunk maps (largest entry), 0 if more
// than kUWinChunks chunks or no interior.  A window's cut enters as a zero state; the error it
// leaves decays as the chunk maps' powers (their spectral radius is the decay rate of the
// inverse's entries), so the rows at least O from a cut differ from the whole system's by
// well below FP64 rounding.
constexpr int kUWinChunks = 64;
constexpr double kUWinTol = 1.3877787807814457e-17;  // 2^-56

__global__ void k_uplan32(F32Tables T, int64_t nfac, const int32_t* __restrict__ shape, float4* __restrict__ urec,
                          int2* __restrict__ uwin) {
  const int64_t s = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (s >= nfac) return;
  const int n = T.n[s];
  const int PT = shape[s] & 0xffff, L = shape[s] >> 16;
  const float* F = T.fac + T.foff[s] * 4;
  auto at = [&](int i, int p) {
    const int tg = i / L, j = i - tg * L;
    return F[((int64_t)(j / 4) * 2 + p) * PT * 4 + (int64_t)tg * 4 + (j & 3)];
  };
  float ia = 0.f, bi = 0.f;
  int K = n;  // no interior
  if (n >= 4) {
    const int c = n - 3;
    ia = at(c, 0);
    bi = at(c, 1);
    K = 0;
    for (int top = c; top >= 0; top -= 32) {  // rows top-31 .. top, from the end
      const int i = top - lane;
      const bool diff = i >= 0 && (at(i, 0) != ia || at(i, 1) != bi);
      const unsigned m = __ballot_sync(kFull, diff);
      if (m) {
        // the differing row nearest the end is the one of the lowest lane with diff set
        K = top - (__ffs(m) - 1) + 1;
        break;
      }
    }
  }
  if (lane != 0) return;
  const double sg = (double)T.sig2[s].x, a = (double)ia, b = (double)bi;
  M2 Mf{1, 0, 0, 1}, Mb{1, 0, 0, 1};
  for (int j = 0; j < L; ++j) {
    Mf = M2{Mf.c, Mf.d, -a * (sg * Mf.a + b * Mf.c), -a * (sg * Mf.b + b * Mf.d)};
    Mb = M2{-a * (b * Mb.a + sg * Mb.c), -a * (b * Mb.b + sg * Mb.d), Mb.a, Mb.b};
  }
  float4* R = urec + s * kURecFloat4;
  int nl[2] = {5, 5};
  bool small[2] = {false, false};
  for (int dir = 0; dir < 2; ++dir) {
    const M2 M = dir == 0 ? Mf : Mb;
    float4* P2 = R + (dir == 0 ? kUFwd2 : kUBwd2);
    float4* PK = R + (dir == 0 ? kUFwdK : kUBwdK);
    M2 p = M;
    for (int l = 0; l < 6; ++l) {  // M^(2^l)
      P2[l] = to_f4(p);
      if (l < 5 && nl[dir] == 5 && norm2(p) < (double)kUTol) nl[dir] = l;
      if (l == 5) small[dir] = norm2(p) < (double)kUTol;
      p = mul2(p, p);
    }
    M2 q{1, 0, 0, 1};
    for (int k = 0; k < 32; ++k) {  // M^k
      PK[k] = to_f4(q);
      q = mul2(M, q);
    }
  }
  const int flags = nl[0] | (nl[1] << 8) | ((int)small[0] << 16) | ((int)small[1] << 17);
  R[0] = make_float4(ia, bi, __int_as_float(K), __int_as_float(flags));
  if (uwin) {
    int O = 0;
    if (K <= n - 3) {
      M2 qf = Mf, qb = Mb;
      for (int k = 1; k <= kUWinChunks; ++k) {
        if (fmax(norm2(qf), norm2(qb)) <= kUWinTol) {
          O = k * L;
          break;
        }
        qf = mul2(Mf, qf);
        qb = mul2(Mb, qb);
      }
    }
    uwin[s] = make_int2(K, O);
  }
}

template <int L, int WT, int REF, int IN, int OUT>
cudaError_t launch_u(const F32Tables& T, const float4* urec, int32_t* kscale, const int32_t* sys, const F32Bucket& b,
                     int shared, const double* f, double* x, cudaStream_t st) {
  const int vec = ((((uintptr_t)f) | ((uintptr_t)x)) % 16 == 0) && b.even_offsets;
  const int W = WT > 0 ? WT : b.W;
  const size_t smem = usmem_bytes(W, L);
  k_solve32u<L, WT, REF, IN, OUT, 0><<<(unsigned)b.count, 32 * W, smem, st>>>(T, urec, kscale, sys + b.first, shared,
                                                                             f, x, vec, W, UWinArgs{});
  return cudaGetLastError();
}

// Grid of a window launch: one CTA per window, or (persistent) as many as stay resident.
template <class K>
cudaError_t window_grid(K kernel, int block, size_t smem, int64_t nwin, bool persistent, unsigned* grid) {
  *grid = (unsigned)nwin;
  if (!persistent) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  if (e != cudaSuccess) return e;
  *grid = (unsigned)std::min<int64_t>(nwin, (int64_t)std::max(per_sm, 1) * sms);
  return cudaSuccess;
}

template <int WT, int REF>
cudaError_t launch_w(const F32Tables& T, const float4* urec, const UWinArgs& wa, int shared, int even_offsets,
                     const double* f, double* x, bool persistent, cudaStream_t st) {
  const int vec = ((((uintptr_t)f) | ((uintptr_t)x)) % 16 == 0) && even_offsets;
  const size_t smem = usmem_bytes(WT, 8);
  if (!persistent) {
    k_solve32u<8, WT, REF, 0, 0, 1><<<(unsigned)wa.nwin, 32 * WT, smem, st>>>(T, urec, nullptr, nullptr, shared, f, x,
                                                                              vec, WT, wa);
    return cudaGetLastError();
  }
  unsigned grid;
  const cudaError_t e = window_grid(k_solve32u<8, WT, REF, 0, 0, 2>, 32 * WT, smem, wa.nwin, true, &grid);
  if (e != cudaSuccess) return e;
  k_solve32u<8, WT, REF, 0, 0, 2><<<grid, 32 * WT, smem, st>>>(T, urec, nullptr, nullptr, shared, f, x, vec, WT, wa);
  return cudaGetLastError();
}

// Copy the overlap rows of every window out of f (before an in-place windowed solve): one warp
// per window, halo[w][0][0 .. O) = rows w0 .. w0 + O - 1 (after a cut at w0), halo[w][1][0 .. O)
// = the window's last O rows (before a cut at its end); row pairs when every windowed system
// starts at an even row (O and the window's first row are multiples of 8).
__global__ void k_uwin_halo(F32Tables T, const int4* __restrict__ win, int64_t nwin, int omax, int pairs,
                            const double* __restrict__ f, double* __restrict__ halo) {
  const int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  if (w >= nwin) return;
  const int lane = threadIdx.x & 31;
  const int4 d = win[w];
  const int n = T.n[d.x], m = d.z & 0xffff, O = d.z >> 16;
  const double* fs = f + T.off[d.x] + d.y;
  double* hb = halo + w * 2 * omax;
  const bool left = d.y > 0, right = d.y + m < n;
  if (pairs) {
    for (int i = lane; i < O / 2; i += 32) {
      if (left) reinterpret_cast<double2*>(hb)[i] = reinterpret_cast<const double2*>(fs)[i];
      if (right) reinterpret_cast<double2*>(hb + omax)[i] = reinterpret_cast<const double2*>(fs + m - O)[i];
    }
  } else {
    for (int i = lane; i < O; i += 32) {
      if (left) hb[i] = fs[i];
      if (right) hb[omax + i] = fs[m - O + i];
    }
  }
}

template <int L, int WT>
cudaError_t dispatch_modes(const F32Tables& T, const float4* urec, int32_t* kscale, const int32_t* sys,
                           const F32Bucket& b, int shared, const double* f, double* x, int max_refine, int in_ff,
                           int out_ff, cudaStream_t st) {
  const int code = (max_refine > 0 ? 4 : 0) | (in_ff ? 2 : 0) | (out_ff ? 1 : 0);
  switch (code) {
    case 0: return launch_u<L, WT, 0, 0, 0>(T, urec, kscale, sys, b, shared, f, x, st);
    case 1: return launch_u<L, WT, 0, 0, 1>(T, urec, kscale, sys, b, shared, f, x, st);
    case 2: return launch_u<L, WT, 0, 1, 0>(T, urec, kscale, sys, b, shared, f, x, st);
    case 3: return launch_u<L, WT, 0, 1, 1>(T, urec, kscale, sys, b, shared, f, x, st);
    case 4: return launch_u<L, WT, 1, 0, 0>(T, urec, kscale, sys, b, shared, f, x, st);
    case 5: return launch_u<L, WT, 1, 0, 1>(T, urec, kscale, sys, b, shared, f, x, st);
    case 6: return launch_u<L, WT, 1, 1, 0>(T, urec, kscale, sys, b, shared, f, x, st);
    default: return launch_u<L, WT, 1, 1, 1>(T, urec, kscale, sys, b, shared, f, x, st);
  }
}

}  // namespace

bool solve32u_supported(const F32Bucket& b) {
  if (b.C != 1) return false;
  if (b.L == 8) return b.W >= 1 && b.W <= 16;
  if (b.L == 4) return b.W == 1;
  return false;
}

cudaError_t launch_uplan32(const F32Tables& T, const int32_t* shape, int64_t nfac, float4* urec, int2* uwin,
                           cudaStream_t st) {
  const int warps = 4;
  k_uplan32<<<(unsigned)((nfac + warps - 1) / warps), 32 * warps, 0, st>>>(T, nfac, shape, urec, uwin);
  return cudaGetLastError();
}

bool solve32w_supported(int W) { return W == 4 || W == 8 || W == 16; }

cudaError_t launch_solve32w(const F32Tables& T, const float4* urec, const int32_t* fshape, const int4* win,
                            int64_t nwin, int W, int omax, int shared, int even_offsets, const double* f, double* x,
                            double* halo, int max_refine, bool persistent, cudaStream_t st) {
  if (nwin == 0) return cudaSuccess;
  if (max_refine > 1 || !solve32w_supported(W) || omax <= 0 || omax % 8) return cudaErrorInvalidValue;
  const bool in_place = f == x;
  if (in_place) {
    const int wpb = 4;  // windows (warps) per CTA
    const int pairs = even_offsets && ((uintptr_t)f) % 16 == 0;
    k_uwin_halo<<<(unsigned)((nwin + wpb - 1) / wpb), 32 * wpb, 0, st>>>(T, win, nwin, omax, pairs, f, halo);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const UWinArgs wa{win, nwin, fshape, in_place ? halo : nullptr, omax};
  const bool r = max_refine > 0;
  switch (W) {
    case 4:
      return r ? launch_w<4, 1>(T, urec, wa, shared, even_offsets, f, x, persistent, st)
               : launch_w<4, 0>(T, urec, wa, shared, even_offsets, f, x, persistent, st);
    case 8:
      return r ? launch_w<8, 1>(T, urec, wa, shared, even_offsets, f, x, persistent, st)
               : launch_w<8, 0>(T, urec, wa, shared, even_offsets, f, x, persistent, st);
    default:
      return r ? launch_w<16, 1>(T, urec, wa, shared, even_offsets, f, x, persistent, st)
               : launch_w<16, 0>(T, urec, wa, shared, even_offsets, f, x, persistent, st);
  }
}

cudaError_t launch_solve32u(const F32Tables& T, const float4* urec, int32_t* kscale, const int32_t* sys,
                            const F32Bucket& b, int shared, const double* f, double* x, int max_refine, int in_ff,
                            int out_ff, cudaStream_t st) {
  if (b.count == 0) return cudaSuccess;
  if (max_refine > 1 || !solve32u_supported(b)) return cudaErrorInvalidValue;
  if (b.L == 4) return dispatch_modes<4, 1>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
  switch (b.W) {
    case 1: return dispatch_modes<8, 1>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
    case 2: return dispatch_modes<8, 2>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
    case 4: return dispatch_modes<8, 4>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
    case 8: return dispatch_modes<8, 8>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
    case 16: return dispatch_modes<8, 16>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
    default:  // the other widths (3, 5-7, 9-15 warps): one kernel for all, compiled for up to 512 threads
      return dispatch_modes<8, 0>(T, urec, kscale, sys, b, shared, f, x, max_refine, in_ff, out_ff, st);
  }
}

}  // namespace pent
