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
//   k_colsweep    in place on rhs^T with the x factors (columns = grid rows);
//   k_transpose   W^T -> W;
//   k_colsweep    in place on W with the y factors, summing dC per column;
//   k_adi_update  C += dC - mean.
#include <cstdint>

#include "internal.cuh"

namespace pent {
namespace {

__device__ __forceinline__ int mirror_idx(int j, int n) {
  while (j < 0 || j >= n) j = (j < 0) ? (-1 - j) : (2 * n - 1 - j);
  return j;
}

constexpr int kTile = 32;      // output tile edge
constexpr int kRowsPerThr = 4;  // block is 32 x 8 threads

// rhs = mu L(C^3 - C) - sigma L(L C) on a 32 x 32 tile, written transposed:
// rhsT[x * ny + y].  C is staged with a two-cell mirrored halo; u = C^3 - C and
// L C are formed on the tile plus a one-cell halo, then both outer Laplacians.
__global__ void __launch_bounds__(256) k_adi_rhs_T(const double* __restrict__ C, double* __restrict__ rhsT, int nx,
                                                  int ny, double mu, double sigma) {
  __shared__ double sC[kTile + 4][kTile + 4 + 1];
  __shared__ double sU[kTile + 2][kTile + 2 + 1];
  __shared__ double sL[kTile + 2][kTile + 2 + 1];
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
      sU[yy][xx] = fma(c * c, c, -c);
      sL[yy][xx] = (sC[yy + 1][xx] + sC[yy + 1][xx + 2]) + (sC[yy][xx + 1] + sC[yy + 2][xx + 1]) - 4.0 * c;
    }
  __syncthreads();
  for (int r = 0; r < kRowsPerThr; ++r) {
    const int yy = ty + 8 * r, xx = tx;
    const double lu = (sU[yy + 1][xx] + sU[yy + 1][xx + 2]) + (sU[yy][xx + 1] + sU[yy + 2][xx + 1]) - 4.0 * sU[yy + 1][xx + 1];
    const double ll = (sL[yy + 1][xx] + sL[yy + 1][xx + 2]) + (sL[yy][xx + 1] + sL[yy + 2][xx + 1]) - 4.0 * sL[yy + 1][xx + 1];
    sO[xx][yy] = fma(mu, lu, -sigma * ll);
  }
  __syncthreads();
  for (int r = 0; r < kRowsPerThr; ++r) {
    const int xx = ty + 8 * r, yy = tx;  // write row xx of the transposed tile: consecutive y
    const int gx = x0 + xx, gy = y0 + yy;
    if (gx < nx && gy < ny) rhsT[(int64_t)gx * ny + gy] = sO[xx][yy];
  }
}

// In place solve down every column of a row-major ncols x n array (element
// (i, col) at buf[i * ncols + col]) with one shared factorisation: thread =
// column, consecutive threads = consecutive addresses.  Forward substitution
// L g = f, then back substitution R x = g (Sec. 2.4), with the FP64 factor
// records of a shared-matrix plan (fwd[i*3+p], bwd[i*2+p], read by every
// thread alike).  With `colsum` every warp (block x 4 + warp) writes the sum
// of its 32 columns of x.
template <int U>
__global__ void __launch_bounds__(128) k_colsweep(double* __restrict__ buf, int ncols, int n,
                                                  const double* __restrict__ fwd, const double* __restrict__ bwd,
                                                  double* colsum) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = col < ncols;
  const int c = active ? col : ncols - 1;
  double g1 = 0.0, g2 = 0.0;
  for (int i0 = 0; i0 < n; i0 += U) {
    double fv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) fv[u] = (i0 + u < n) ? buf[(int64_t)(i0 + u) * ncols + c] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u;
      if (i < n) {
        const double g = fma(-__ldg(fwd + i * 3 + 1), g1, fma(-__ldg(fwd + i * 3 + 2), g2, __ldg(fwd + i * 3) * fv[u]));
        if (active) buf[(int64_t)i * ncols + c] = g;
        g2 = g1;
        g1 = g;
      }
    }
  }
  double x1 = 0.0, x2 = 0.0, sum = 0.0;
  for (int i0 = n - 1; i0 >= 0; i0 -= U) {
    double gv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) gv[u] = (i0 - u >= 0) ? buf[(int64_t)(i0 - u) * ncols + c] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 - u;
      if (i >= 0) {
        const double xv = fma(-__ldg(bwd + i * 2), x1, fma(-__ldg(bwd + i * 2 + 1), x2, gv[u]));
        if (active) buf[(int64_t)i * ncols + c] = xv;
        sum += xv;
        x2 = x1;
        x1 = xv;
      }
    }
  }
  if (colsum) {  // one partial sum per warp, in a fixed order (deterministic mean)
    if (!active) sum = 0.0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if ((threadIdx.x & 31) == 0) colsum[(blockIdx.x * blockDim.x + threadIdx.x) >> 5] = sum;
  }
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

// C += dC - mean(dC), mean = (sum of the per-warp column sums) / count, summed
// in the same order by every block.
__global__ void __launch_bounds__(256) k_adi_update(double* __restrict__ C, const double* __restrict__ dC,
                                                    const double* __restrict__ colsum, int nparts, double inv_count,
                                                    int64_t count) {
  __shared__ double s_mean;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < nparts; ++k) t += colsum[k];
    s_mean = t * inv_count;
  }
  __syncthreads();
  const double mean = s_mean;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += stride) C[i] += dC[i] - mean;
}

}  // namespace

cudaError_t launch_adi_step(const AdiArgs& a, cudaStream_t st) {
  const dim3 blk(32, 8);
  const dim3 grd((a.nx + kTile - 1) / kTile, (a.ny + kTile - 1) / kTile);
  k_adi_rhs_T<<<grd, blk, 0, st>>>(a.C, a.rhsT, a.nx, a.ny, a.mu, a.sigma);
  // x sweep: columns of rhs^T are the grid rows (ny systems of n = nx)
  k_colsweep<8><<<(a.ny + 127) / 128, 128, 0, st>>>(a.rhsT, a.ny, a.nx, a.fx.fwd, a.fx.bwd, nullptr);
  k_transpose<<<dim3((a.ny + kTile - 1) / kTile, (a.nx + kTile - 1) / kTile), blk, 0, st>>>(a.rhsT, a.W, a.nx, a.ny);
  // y sweep: columns of W are the grid columns (nx systems of n = ny); one partial sum per warp
  const int blocks = (a.nx + 127) / 128;
  k_colsweep<8><<<blocks, 128, 0, st>>>(a.W, a.nx, a.ny, a.fy.fwd, a.fy.bwd, a.colsum);
  const int64_t count = (int64_t)a.nx * a.ny;
  k_adi_update<<<4 * 152, 256, 0, st>>>(a.C, a.W, a.colsum, blocks * 4, 1.0 / (double)count, count);
  return cudaGetLastError();
}

}  // namespace pent
