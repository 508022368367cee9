// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pent {

constexpr int kWarp = 32;

// Device info word (int64 x 4):
//   [0] lowest (system << 32 | row) whose pivot failed, or kInfoNone
//   [1] largest number of refinement steps any system used
//   [2] flags: bit 0 = refinement not converged
//   [3] unused
constexpr int kInfoWords = 4;
constexpr unsigned long long kInfoNone = 0x7f7f7f7f7f7f7f7full;  // every byte 0x7f: settable by cudaMemsetAsync

// Read-only view of the plan's per-system tables and factor storage, passed by value to kernels.
struct DevPlan {
  int64_t batch;        // number of systems
  int64_t ngroups;      // ceil(batch / 32): one group of 32 systems per warp in thread-per-system kernels
  int shared;           // all systems share one matrix
  int64_t n_shared;     // rows of the shared matrix
  const int32_t* perm;  // [ngroups*32] system at sorted position q (-1 for padding lanes)
  const int64_t* off;   // [batch] first row of each system in the caller's layout
  const int32_t* n;     // [batch] rows of each system
  const int64_t* goff;  // [ngroups] first record row of each group
  const int32_t* glen;  // [ngroups] padded rows of each group (max n in the group)
  unsigned long long* info;
};

// FP64 factor records, per group of 32 systems and row r (record row R = goff[k] + r),
// stored in row pairs (see core64.cu):
//   general band:   fwd planes p = 0: 1/alpha, 1: beta/alpha, 2: epsilon/alpha
//   hyperdiffusion: fwd planes p = 0: 1/alpha, 1: beta (epsilon_i = sigma_s for every
//                   row i >= 2, so it is not stored; padding rows have 1/alpha = 0)
//   bwd planes p = 0: gamma, 1: delta
// For a shared matrix (always the general form): fwd[r*3 + p], bwd[r*2 + p].
struct F64Factors {
  double* fwd;
  double* bwd;
  const double* sig;  // per-system sigma of hyperdiffusion records, nullptr for the general form
  // Hyperdiffusion records only (or nullptr): per group lane q = 32 k + lane the records of an interior
  // row pair, icst[4 q + p] for plane p = 1/alpha, beta, gamma, delta (a double2 of the pair's rows),
  // the same bits on every pair ik[q] .. (n - 4) / 2 of the lane's system (ik[q] = INT_MAX: none),
  // which the walks then take from registers instead of memory.
  const double2* icst = nullptr;
  const int32_t* ik = nullptr;
};

// FP32 storage of the symmetric hyperdiffusion factors, one block per system s
// (P T = 32 W C threads of L rows, n_s <= P T L): float4 T.foff[s] + ((j / 4) * 2 + p) * P T + t
// holds rows t L + 4 (j/4) .. + 3 of plane p (0: 1/alpha, 1: beta); epsilon, gamma and
// delta are rebuilt from sigma in the solve.  Shared-matrix plans use block 0.
struct F32Tables {
  const int32_t* n;       // [batch] rows
  const int64_t* off;     // [batch] first row in f / x
  const int64_t* foff;    // [nfac] first float4 of the factor block
  float2* sig2;           // [nfac] sigma split into an FP32 pair (hi, lo)
  const double* sigma;    // [nfac] sigma in FP64 (FP64-residual variant)
  float* fac;             // factor storage
  unsigned long long* info;
  float4* psinv;          // [nfac] periodic plans: S^{-1} of Navon's reduction (row-major 2 x 2)
};

// Systems solved by one launch: sys[first .. first + count) share the CTA shape
// (L rows per thread, W warps per CTA, C CTAs per system in a cluster).
struct F32Bucket {
  int L, W, C;
  int64_t first, count;
  int even_offsets;  // every system of the bucket starts at an even row (16-byte vector access)
};

// Partitioned FP64 solve of groups whose systems are long: each group's rows are
// cut into chunks of kLongChunk rows, one warp per (group, chunk), joined by
// per-lane scans over the chunks (csrc/core64.cu).
constexpr int kLongChunk = 256;  // even: chunks hold whole row pairs
struct F64Part {
  const int32_t* ck;     // [nchunks] group of each chunk (chunks of a group are consecutive)
  const int32_t* cc;     // [nchunks] index of the chunk within its group
  const int64_t* cbase;  // [ngroups] first chunk of each partitioned group
  const int32_t* cnum;   // [ngroups] chunks of each partitioned group (0 otherwise)
  double* cmap;          // [nchunks][8][32]: forward (0..3) and back (4..7) 2x2 maps per lane
  double2* U;            // [nchunks][32] affine parts
  double2* E;            // [nchunks][32] entering states
};

// Periodic (cyclic) systems by Navon's reduction (csrc/periodic.cu).  Every
// per-row array of the reduced matrix E (m = n - 2 rows) is interleaved,
// p[r * S + s] with S = batch, or p[r] when the matrix is shared.
struct PerArgs {
  int64_t batch, n, m;
  int shared;
  double *ia, *bb, *ee;  // 1/alpha, beta/alpha, epsilon/alpha of E
  double *ga, *de;       // gamma, delta of E
  double *z0, *z1;       // Z = E^{-T} h (h^T: rows n-2, n-1 of A in columns 0..m-1)
  double *w0, *w1;       // W = L^{-1} k (k: columns n-2, n-1 of A in rows 0..m-1)
  double* sinv;          // [S][4] inverse of S = D - h^T E^{-1} k, row-major
  double* gscr;          // [m][batch] forward scratch g
  unsigned long long* info;
};

// ---- launchers (kernels live in the .cu files) ----
cudaError_t launch_factor64(const DevPlan& P, const double* a, const double* b, const double* c, const double* d,
                            const double* e, const double* sigma, F64Factors F, cudaStream_t st);
cudaError_t launch_factor32(const F32Tables& T, const int32_t* shape, int64_t nsys, const double* sigma,
                            cudaStream_t st);
// Groups [g0, g1) of the plan (all of them for a shared matrix: g0 = 0, g1 = ngroups).
cudaError_t launch_solve64(const DevPlan& P, F64Factors F, const double* f, double* x, double* gscr, int block_warps,
                           int unroll, int64_t g0, int64_t g1, cudaStream_t st);
// Chunk maps of chunks [c0, c1) (after the factorisation), and the partitioned
// solve of groups [kbeg, kend) whose chunks are [c0, c1).
cudaError_t launch_chunk_maps64(const DevPlan& P, F64Factors F, const F64Part& X, int64_t c0, int64_t c1,
                                cudaStream_t st);
cudaError_t launch_solve64_part(const DevPlan& P, F64Factors F, const F64Part& X, const double* f, double* x,
                                double* gscr, int64_t kbeg, int64_t kend, int64_t c0, int64_t c1, cudaStream_t st);
// One time step in place on C with f = C + mu_s D2(C^3 - C) - nu_s D4 C assembled in the
// forward sweep (hyperdiffusion records, groups [g0, g1)); and the same f written out to
// `f` for the systems of groups [g0, g1) (used before the partitioned solve).
cudaError_t launch_step64(const DevPlan& P, F64Factors F, const double* mu, const double* nu, double* C,
                          double* gscr, int block_warps, int unroll, int64_t g0, int64_t g1, cudaStream_t st);
cudaError_t launch_step_rhs(const DevPlan& P, const double* mu, const double* nu, const double* C, double* f,
                            int64_t g0, int64_t g1, cudaStream_t st);
// Factor A_s = I + sigma_s D4 (hyperdiffusion records, sigma copied into F.sig) and solve
// A_s x = f in one pass per system, groups [g0, g1).
cudaError_t launch_refactor_solve64(const DevPlan& P, F64Factors F, const double* sigma, const double* f, double* x,
                                    double* gscr, int block_warps, int64_t g0, int64_t g1, cudaStream_t st);
// Interior records of hyperdiffusion factorisations (F.icst, F.ik; csrc/core64.cu).
cudaError_t launch_interior64(const DevPlan& P, F64Factors F, double2* icst, int32_t* ik, cudaStream_t st);
// Windowed walks of groups of long hyperdiffusion systems (csrc/core64.cu).  gover: per group the
// overlap rows a window needs (a multiple of 8; 0x7fff: more than omax).  win: per window (group,
// first row, rows | overlap << 16); side: [nwin][omax / 2][32] double2 of g after the kept rows;
// halo: [nwin][2][omax / 2][32] double2 of overlap rows, filled first when f == x.
cudaError_t launch_overlap64(const DevPlan& P, F64Factors F, int omax, int32_t* gover, int32_t* lover, cudaStream_t st);
// system windows (one window per thread): the per-system record copy, then both walks
cudaError_t launch_srec64(const DevPlan& P, F64Factors F, const int32_t* wg, int64_t nwg, int64_t max_pairs,
                          const int64_t* sbase, double2* sfwd, double2* sbwd, cudaStream_t st);
cudaError_t launch_swin64(const DevPlan& P, F64Factors F, const int4* win, int64_t nwin, int window_rows, int unroll,
                          int block_warps, const double2* sfwd, const double2* sbwd, const int64_t* sbase,
                          const double* f, double* x, double2* gs, cudaStream_t st);
// persistent: a grid of as many CTAs as stay resident, whose warps take the windows in turn.
cudaError_t launch_solve64w(const DevPlan& P, F64Factors F, const int4* win, int64_t nwin, int omax, int unroll,
                            int block_warps, const double* f, double* x, double* gscr, double* side, double* halo,
                            bool persistent, cudaStream_t st);
cudaError_t launch_adjoint64(const DevPlan& P, F64Factors F, const double* f, double* x, double* gscr,
                             int block_warps, cudaStream_t st);
// step: f is the field C and the kernel assembles the right-hand side C + mu D2(C^3 - C) - nu D4 C
// (float-float) before the solve (pent_step_batch); mu, nu per factored system, or NULL.
cudaError_t launch_solve32r(const F32Tables& T, const int32_t* sys, const F32Bucket& b, int shared, const double* f,
                            double* x, int max_refine, int residual_f64, int tol_log2, cudaStream_t st,
                            const double* mu = nullptr, const double* nu = nullptr, bool step = false,
                            bool periodic = false);
// FP32 hyperdiffusion plans, interior-constant kernel (csrc/f32u.cu).  Per factor block a record of
// kURecFloat4 float4: (1/alpha, beta of the interior, K = first row of the interior, scan levels and
// flags), then the powers M^(2^l) (l = 0..5) and M^k (k = 0..31) of the forward and of the back
// chunk map.  kscale: per system, the power of two by which a field kept as float pairs is scaled.
constexpr int kURecFloat4 = 77;
// uwin (or nullptr): per factor block (K, O), O the overlap rows of a window of the system (0: none
// keeps the windowed solve within FP64 rounding of the whole system's).
cudaError_t launch_uplan32(const F32Tables& T, const int32_t* shape, int64_t nfac, float4* urec, int2* uwin,
                           cudaStream_t st);
// True if the bucket's CTA shape has an instantiation of the interior-constant kernel.
bool solve32u_supported(const F32Bucket& b);
// in_ff / out_ff: f / x hold float pairs (h, l) per row scaled by 2^-kscale[s] instead of FP64
// values (x may alias f); max_refine 0 or 1.
cudaError_t launch_solve32u(const F32Tables& T, const float4* urec, int32_t* kscale, const int32_t* sys,
                            const F32Bucket& b, int shared, const double* f, double* x, int max_refine, int in_ff,
                            int out_ff, cudaStream_t st);
// Windowed solve of long systems (csrc/f32u.cu): CTA k of W warps (8 rows a thread) solves window
// win[k] = (system, first row, rows | overlap rows << 16) and writes the rows at least the overlap
// from its cuts; fshape: each factor block's threads | L << 16.  An in-place solve (f == x) first
// copies the overlap rows into halo ([nwin][2][omax] doubles).  max_refine 0 or 1.
bool solve32w_supported(int W);
// persistent: a grid of as many CTAs as stay resident, which take the windows in turn.
cudaError_t launch_solve32w(const F32Tables& T, const float4* urec, const int32_t* fshape, const int4* win,
                            int64_t nwin, int W, int omax, int shared, int even_offsets, const double* f, double* x,
                            double* halo, int max_refine, bool persistent, cudaStream_t st);
// Periodic FP32 plans: factors of E, the columns of Z = E^{-1} k and S^{-1} (k_factor32_periodic).
cudaError_t launch_factor32_periodic(const F32Tables& T, const int32_t* shape, int64_t nsys, const double* sigma,
                                     cudaStream_t st);
cudaError_t launch_factor_periodic(const PerArgs& A, const double* a, const double* b, const double* c,
                                   const double* d, const double* e, const double* sigma, cudaStream_t st);
// rhs: assemble f_i = C_i + mu_s (D2 (C^3 - C))_i - nu_s (D4 C)_i from the field in f (periodic stencils).
cudaError_t launch_solve_periodic(const PerArgs& A, const double* f, double* x, const double* mu, const double* nu,
                                  bool rhs, cudaStream_t st);
cudaError_t launch_sigma_grad(const DevPlan& P, const double* mu, const double* x, double* g_sigma, cudaStream_t st);
// Rows per chunk of the partitioned column sweeps of the ADI step.
constexpr int kAdiChunk = 64;

// Scratch of one partitioned sweep of `ncols` columns of n rows (nchunks = ceil(n / kAdiChunk)).
struct SweepArgs {
  F64Factors f;        // shared-matrix records (n rows)
  const double* cmap;  // [nchunks][8] chunk maps (k_chunk_maps)
  double2* U;          // [nchunks][ncols] affine parts
  double2* E;          // [nchunks][ncols] entering states
};

// One ADI step (csrc/adi.cu).  rhsT and W are field-sized scratch; parts holds
// ceil(nx / 32) * ceil(ny / kAdiChunk) partial sums and mean one double.
struct AdiArgs {
  double* C;
  double* rhsT;
  double* W;
  double* parts;
  double* mean;
  int nx, ny;
  double mu, sigma;
  SweepArgs sx;  // x sweep: I + sigma D4 with n = nx, ny columns
  SweepArgs sy;  // y sweep: n = ny, nx columns
};
cudaError_t launch_adi_step(const AdiArgs& a, cudaStream_t st);
// dst[0 .. count) = v on stream st.
cudaError_t launch_fill(double* dst, double v, int64_t count, cudaStream_t st);
// Chunk maps of a shared FP64 factorisation with n rows (once per factorisation).
cudaError_t launch_chunk_maps(F64Factors F, int n, double* cmap, cudaStream_t st);

}  // namespace pent
