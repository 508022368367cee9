// Two-dimensional Cahn-Hilliard step by alternating directions (ADI).
//
// The paper names ADI as the way its batched pentadiagonal solver carries over
// to 2D (Sec. 4, citing Douglas 1955) without giving a scheme; this file
// implements the Douglas delta form of the semi-implicit step of Sec. 2.1
// (D = 1) on an ny x nx grid with no-flux walls:
//   rhs = mu L(C^3 - C) - sigma L(L C),        mu = dt/dx^2, sigma = gamma dt/dx^4,
//   (I + sigma D4_x) W = rhs                   (one system per grid row, n = nx)
//   (I + sigma D4_y) dC = W                    (one system per grid column, n = ny)
//   C <- C + dC - mean(dC).
// L is the five-point Laplacian; every ghost value mirrors the cell next to the
// wall, the same reflection as the hyperdiffusion band, so D4 = D2N^2 in each
// direction.  Exact dC has zero mean (L has zero column sums, each implicit
// factor unit column sums); removing the mean of the computed dC keeps the
// total mass to the rounding of C itself.
//
// Data flow of one step (all FP64, field in L2 for 2048^2):
//   k_adi_rhs_T   C -> rhs, written transposed (x-major), so that the x sweep
//                 becomes a column sweep with coalesced access;
//   x sweep       in place on rhs^T with the x factors (columns = grid rows);
//   k_transpose   W^T -> W;
//   y sweep       in place on W with the y factors, summing dC per chunk;
//   k_sum_parts   the mean of dC, summed in a fixed order;
//   k_adi_update  C += dC - mean.
// Each sweep is partitioned: every column is cut into chunks of kChunk rows,
// one thread per (column, chunk).  A substitution is a second-order linear
// recurrence, so a chunk maps the two values carried into it affinely; the
// linear part depends on the (shared) factors only and is computed once per
// factorisation (k_chunk_maps).  A zero-state pass gives each chunk's affine
// part, a short scan per column over the chunks gives every chunk's entering
// state, and a second pass from it produces the result.  This keeps 32x more
// threads busy than a thread-per-column sweep.
#include <cstdint>

#include "internal.cuh"

namespace pent {
namespace {

__device__ __forceinline__ int mirror_idx(int j, int n) {
  while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
  return j;
}

constexpr int kTile = 32;      // output tile edge
constexpr int kChunk = kAdiChunk;
constexpr int kRowsPerThr = 4;  // block is 32 x 8 threads

// rhs = mu L(C^3 - C) - sigma L(L C) on a 32 x 32 tile, written transposed:
// rhsT[x * ny + y].  L is linear, so this is L w with w = mu (C^3 - C) - sigma L C:
// C is staged with a two-cell mirrored halo, w is formed on the tile plus a
// one-cell halo (the even reflection commutes with L, so w's halo is the
// reflection of w), then one outer Laplacian -- a quarter fewer FP64 operations
// than two outer Laplacians, on a kernel bound by the FP64 pipe.
__global__ void __launch_bounds__(256) k_adi_rhs_T(const double* __restrict__ C, double* __restrict__ rhsT, int nx,
                                                  int ny, double mu, double sigma) {
  __shared__ double sC[kTile + 4][kTile + 4 + 1];
  __shared__ double sW[kTile + 2][kTile + 2 + 1];
  __shared__ double sO[kTile][kTile + 1];
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < kTile + 4; yy += 8)
    for (int xx = tx; xx < kTile + 4; xx += 32) {
      const int gy = mirror_idx(y0 + yy - 2, ny), gx = mirror_idx(x0 + xx - 2, nx);
      sC[yy][xx] = C[(int64_t)gy * nx + gx];
    }
  __syncthreads();
  for (int yy = ty; yy < kTile + 2; yy += 8)
    for (int xx = tx; xx < kTile + 2; xx += 32) {
      const double c = sC[yy + 1][xx + 1];
      const double lc = (sC[yy + 1][xx] + sC[yy + 1][xx + 2]) + (sC[yy][xx + 1] + sC[yy + 2][xx + 1]) - 4.0 * c;
      sW[yy][xx] = fma(mu, fma(c * c, c, -c), -sigma * lc);
    }
  __syncthreads();
  for (int r = 0; r < kRowsPerThr; ++r) {
    const int yy = ty + 8 * r, xx = tx;
    sO[xx][yy] = (sW[yy + 1][xx] + sW[yy + 1][xx + 2]) + (sW[yy][xx + 1] + sW[yy + 2][xx + 1]) - 4.0 * sW[yy + 1][xx + 1];
  }
  __syncthreads();
  for (int r = 0; r < kRowsPerThr; ++r) {
    const int xx = ty + 8 * r, yy = tx;  // write row xx of the transposed tile: consecutive y
    const int gx = x0 + xx, gy = y0 + yy;
    if (gx < nx && gy < ny) rhsT[(int64_t)gx * ny + gy] = sO[xx][yy];
  }
}

// ---- partitioned column sweeps (shared factors, general records fwd[r*3+p], bwd[r*2+p]) ----

// Forward and back maps of every chunk: fwd on (g_{r0-2}, g_{r0-1}) -> (g_{r1-2},
// g_{r1-1}) with g_i = -E_i g_{i-2} - B_i g_{i-1} (+ A_i f_i); back on (x_{r1},
// x_{r1+1}) -> (x_{r0}, x_{r0+1}) with x_i = -gamma_i x_{i+1} - delta_i x_{i+2}
// (+ g_i).  cmap[k*8 + 0..3] forward (row-major 2x2), [k*8 + 4..7] back.  One
// thread per chunk.
__global__ void k_chunk_maps(const double* __restrict__ fwd, const double* __restrict__ bwd, int n, int nchunks,
                             double* __restrict__ cmap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nchunks) return;
  const int r0 = k * kChunk, r1 = min(n, r0 + kChunk);
  double f00 = 1.0, f01 = 0.0, f10 = 0.0, f11 = 1.0;  // rows of the map as they pass each row
  for (int i = r0; i < r1; ++i) {
    const double B = fwd[i * 3 + 1], E = fwd[i * 3 + 2];
    const double n10 = -E * f00 - B * f10, n11 = -E * f01 - B * f11;
    f00 = f10;
    f01 = f11;
    f10 = n10;
    f11 = n11;
  }
  double b00 = 1.0, b01 = 0.0, b10 = 0.0, b11 = 1.0;
  for (int i = r1 - 1; i >= r0; --i) {
    const double G = bwd[i * 2], D = bwd[i * 2 + 1];
    const double n00 = -G * b00 - D * b10, n01 = -G * b01 - D * b11;
    b10 = b00;
    b11 = b01;
    b00 = n00;
    b01 = n01;
  }
  double* m = cmap + (size_t)k * 8;
  m[0] = f00; m[1] = f01; m[2] = f10; m[3] = f11;
  m[4] = b00; m[5] = b01; m[6] = b10; m[7] = b11;
}

struct ChunkIdx {
  int col, k, r0, r1;
  bool active;
};
__device__ __forceinline__ ChunkIdx chunk_idx(int ncols, int n) {
  ChunkIdx c;
  c.col = blockIdx.x * 32 + threadIdx.x;
  c.k = blockIdx.y * blockDim.y + threadIdx.y;
  c.r0 = c.k * kChunk;
  c.r1 = min(n, c.r0 + kChunk);
  c.active = c.col < ncols && c.r0 < n;
  return c;
}

// Forward pass over a chunk from entering state (p2, p1); WRITE stores g in place.
template <bool WRITE>
__device__ __forceinline__ void chunk_fwd(double* __restrict__ buf, int ncols, const ChunkIdx& c,
                                          const double* __restrict__ fwd, double& p2, double& p1) {
  constexpr int U = 8;
  for (int i0 = c.r0; i0 < c.r1; i0 += U) {
    double fv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) fv[u] = (i0 + u < c.r1) ? buf[(int64_t)(i0 + u) * ncols + c.col] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u;
      if (i < c.r1) {
        const double g = fma(-__ldg(fwd + i * 3 + 1), p1, fma(-__ldg(fwd + i * 3 + 2), p2, __ldg(fwd + i * 3) * fv[u]));
        if (WRITE) buf[(int64_t)i * ncols + c.col] = g;
        p2 = p1;
        p1 = g;
      }
    }
  }
}

// Back pass over a chunk from entering state (s1, s2) = (x_{r1}, x_{r1+1});
// WRITE stores x in place and returns the sum of the chunk's x.
template <bool WRITE>
__device__ __forceinline__ double chunk_bwd(double* __restrict__ buf, int ncols, const ChunkIdx& c,
                                            const double* __restrict__ bwd, double& s1, double& s2) {
  constexpr int U = 8;
  double sum = 0.0;
  for (int i0 = c.r1 - 1; i0 >= c.r0; i0 -= U) {
    double gv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) gv[u] = (i0 - u >= c.r0) ? buf[(int64_t)(i0 - u) * ncols + c.col] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 - u;
      if (i >= c.r0) {
        const double xv = fma(-__ldg(bwd + i * 2), s1, fma(-__ldg(bwd + i * 2 + 1), s2, gv[u]));
        if (WRITE) buf[(int64_t)i * ncols + c.col] = xv;
        sum += xv;
        s2 = s1;
        s1 = xv;
      }
    }
  }
  return sum;
}

// Pass 1: forward from a zero state; U[k * ncols + col] = (g_{r1-2}, g_{r1-1}).
__global__ void __launch_bounds__(256) k_psweep_fwd0(double* __restrict__ buf, int ncols, int n,
                                                     const double* __restrict__ fwd, double2* __restrict__ U) {
  const ChunkIdx c = chunk_idx(ncols, n);
  if (!c.active) return;
  double p2 = 0.0, p1 = 0.0;
  chunk_fwd<false>(buf, ncols, c, fwd, p2, p1);
  U[(int64_t)c.k * ncols + c.col] = make_double2(p2, p1);
}

// Entering states of every chunk of a column (thread per column), in sweep
// order: e = 0 at the system's edge, then e <- M_k e + U_k.
template <bool FWD>
__global__ void k_pscan(int ncols, int nchunks, const double* __restrict__ cmap, const double2* __restrict__ U,
                        double2* __restrict__ E) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  double e0 = 0.0, e1 = 0.0;
  for (int j = 0; j < nchunks; ++j) {
    const int k = FWD ? j : nchunks - 1 - j;
    E[(int64_t)k * ncols + col] = make_double2(e0, e1);
    const double* m = cmap + (size_t)k * 8 + (FWD ? 0 : 4);
    const double2 u = U[(int64_t)k * ncols + col];
    const double n0 = fma(m[0], e0, fma(m[1], e1, u.x));
    const double n1 = fma(m[2], e0, fma(m[3], e1, u.y));
    e0 = n0;
    e1 = n1;
  }
}

// Pass 2: forward from the true entering state (g in place), then the back pass
// from a zero state; U[k * ncols + col] = (x_{r0}, x_{r0+1}) of that pass.
__global__ void __launch_bounds__(256) k_psweep_mid(double* __restrict__ buf, int ncols, int n,
                                                    const double* __restrict__ fwd, const double* __restrict__ bwd,
                                                    const double2* __restrict__ Ef, double2* __restrict__ U) {
  const ChunkIdx c = chunk_idx(ncols, n);
  if (!c.active) return;
  const double2 e = Ef[(int64_t)c.k * ncols + c.col];
  double p2 = e.x, p1 = e.y;
  chunk_fwd<true>(buf, ncols, c, fwd, p2, p1);
  double s1 = 0.0, s2 = 0.0;
  chunk_bwd<false>(buf, ncols, c, bwd, s1, s2);
  U[(int64_t)c.k * ncols + c.col] = make_double2(s1, s2);
}

// Pass 3: back pass from the true entering state (x in place).  With `parts`,
// each warp (32 columns of one chunk) writes the sum of its x to
// parts[k * ceil(ncols / 32) + blockIdx.x].
__global__ void __launch_bounds__(256) k_psweep_bwd(double* __restrict__ buf, int ncols, int n,
                                                    const double* __restrict__ bwd, const double2* __restrict__ Eb,
                                                    double* __restrict__ parts) {
  const ChunkIdx c = chunk_idx(ncols, n);
  double sum = 0.0;
  if (c.active) {
    const double2 e = Eb[(int64_t)c.k * ncols + c.col];
    double s1 = e.x, s2 = e.y;
    sum = chunk_bwd<true>(buf, ncols, c, bwd, s1, s2);
  }
  if (parts && c.r0 < n) {  // the whole warp shares c.k, so it agrees on this test
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (threadIdx.x == 0) parts[(int64_t)c.k * gridDim.x + blockIdx.x] = sum;
  }
}

// The sum of nparts partial sums in a fixed order (one block): thread t adds
// parts t, t + 256, ..., then a fixed tree.  out[0] = sum * scale.
__global__ void __launch_bounds__(256) k_sum_parts(const double* __restrict__ parts, int64_t nparts, double scale,
                                                   double* __restrict__ out) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < nparts; i += 256) t += parts[i];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

// out[x * ny + y] -> out2[y * nx + x] (tiled transpose of a ny-column, nx-row array).
__global__ void __launch_bounds__(256) k_transpose(const double* __restrict__ in, double* __restrict__ out, int rows,
                                                   int cols) {
  __shared__ double t[kTile][kTile + 1];
  const int c0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
  for (int r = threadIdx.y; r < kTile; r += 8) {
    const int gr = r0 + r, gc = c0 + threadIdx.x;
    if (gr < rows && gc < cols) t[r][threadIdx.x] = in[(int64_t)gr * cols + gc];
  }
  __syncthreads();
  for (int c = threadIdx.y; c < kTile; c += 8) {
    const int gc = c0 + c, gr = r0 + threadIdx.x;
    if (gr < rows && gc < cols) out[(int64_t)gc * rows + gr] = t[threadIdx.x][c];
  }
}

// C += dC - mean(dC).
__global__ void __launch_bounds__(256) k_adi_update(double* __restrict__ C, const double* __restrict__ dC,
                                                    const double* __restrict__ mean, int64_t count) {
  const double m = *mean;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) C[i] += dC[i] - m;
}

// In place solve of the ncols columns of buf (n rows) with the shared factors
// of s; parts (or nullptr) receives per-warp partial sums of the solution.
cudaError_t sweep(double* buf, int ncols, int n, const SweepArgs& s, double* parts, cudaStream_t st) {
  const int nchunks = (n + kChunk - 1) / kChunk;
  const dim3 blk(32, 8);
  const dim3 grd((ncols + 31) / 32, (nchunks + 7) / 8);
  const int sb = 128, sg = (ncols + sb - 1) / sb;
  k_psweep_fwd0<<<grd, blk, 0, st>>>(buf, ncols, n, s.f.fwd, s.U);
  k_pscan<true><<<sg, sb, 0, st>>>(ncols, nchunks, s.cmap, s.U, s.E);
  k_psweep_mid<<<grd, blk, 0, st>>>(buf, ncols, n, s.f.fwd, s.f.bwd, s.E, s.U);
  k_pscan<false><<<sg, sb, 0, st>>>(ncols, nchunks, s.cmap, s.U, s.E);
  k_psweep_bwd<<<grd, blk, 0, st>>>(buf, ncols, n, s.f.bwd, s.E, parts);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chunk_maps(F64Factors F, int n, double* cmap, cudaStream_t st) {
  const int nchunks = (n + kChunk - 1) / kChunk;
  k_chunk_maps<<<(nchunks + 63) / 64, 64, 0, st>>>(F.fwd, F.bwd, n, nchunks, cmap);
  return cudaGetLastError();
}

cudaError_t launch_adi_step(const AdiArgs& a, cudaStream_t st) {
  const dim3 blk(32, 8);
  const dim3 grd((a.nx + kTile - 1) / kTile, (a.ny + kTile - 1) / kTile);
  k_adi_rhs_T<<<grd, blk, 0, st>>>(a.C, a.rhsT, a.nx, a.ny, a.mu, a.sigma);
  // x sweep: columns of rhs^T are the grid rows (ny systems of n = nx)
  cudaError_t e = sweep(a.rhsT, a.ny, a.nx, a.sx, nullptr, st);
  if (e != cudaSuccess) return e;
  k_transpose<<<dim3((a.ny + kTile - 1) / kTile, (a.nx + kTile - 1) / kTile), blk, 0, st>>>(a.rhsT, a.W, a.nx, a.ny);
  // y sweep: columns of W are the grid columns (nx systems of n = ny), with partial sums of dC
  e = sweep(a.W, a.nx, a.ny, a.sy, a.parts, st);
  if (e != cudaSuccess) return e;
  const int64_t count = (int64_t)a.nx * a.ny;
  const int64_t nparts = (int64_t)((a.nx + 31) / 32) * ((a.ny + kChunk - 1) / kChunk);
  k_sum_parts<<<1, 256, 0, st>>>(a.parts, nparts, 1.0 / (double)count, a.mean);
  k_adi_update<<<4 * 152, 256, 0, st>>>(a.C, a.W, a.mean, count);
  return cudaGetLastError();
}

// dst[0 .. count) = v (a kernel argument: asynchronous and capture-safe, unlike a copy from host memory).
__global__ void k_fill(double* dst, double v, int64_t count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) dst[i] = v;
}

cudaError_t launch_fill(double* dst, double v, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_fill<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(dst, v, count);
  return cudaGetLastError();
}

}  // namespace pent
