/*
 * pentbatch -- batched pentadiagonal factor-once / solve-many on one GB300 GPU.
 *
 * The method is the one of Gloster, O Naraigh and Pang, "cuPentBatch -- A
 * batched pentadiagonal solver for NVIDIA GPUs" (arXiv 1807.07382): each
 * system's matrix A = L R is factorised once without pivoting (Sec. 2.4,
 * factorisation steps 1-14) and kept on the device; every later right-hand
 * side then costs one forward substitution L g = f and one back substitution
 * R x = g (Sec. 2.4, the steps for g and for x; the factor/solve split of
 * Sec. 2.6).  The right-hand sides come from implicit hyperdiffusion steps
 * (Sec. 2.2-2.3) and from alternating-direction steps of the 2D
 * Cahn-Hilliard equation (Sec. 2.1 and the ADI remark of Sec. 4).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  * Rows.  System s has n_s rows; row i (0-based, the paper's row i+1) of
 *    system s is element off[s] + i of every per-row array, with
 *    off[s] = n_0 + ... + n_{s-1} ("system-major" layout).  The library's own
 *    layouts (interleaved, chunked) are private to the workspace.
 *  * Band.  Row i reads a_i x_{i-2} + b_i x_{i-1} + c_i x_i + d_i x_{i+1}
 *    + e_i x_{i+2} (Sec. 2.4, the general pentadiagonal A).  Entries that would
 *    fall outside the matrix (a_0, a_1, b_0, d_{n-1}, e_{n-2}, e_{n-1}) are
 *    never read.
 *  * Memory.  Every pointer argument named d_* or documented as "device" is
 *    device memory owned by the caller.  The library allocates no device
 *    memory: the plan's workspace is caller-provided (pent_plan_bind).
 *  * Asynchrony.  Every call except pent_plan_create/destroy, pent_plan_bind
 *    and pent_get_info is asynchronous on the plan's bound stream, performs no
 *    host synchronisation, allocation or host read-back, and may therefore be
 *    captured into a CUDA graph.
 *  * Errors.  Argument errors are detected on the host before anything is
 *    launched and return PENT_EINVAL.  Numerical failures found on the device
 *    (a zero or non-finite pivot, refinement that does not converge) are
 *    recorded in a device info word and returned by pent_get_info.  Nothing
 *    traps, aborts or throws.
 */
#ifndef PENTBATCH_H
#define PENTBATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PENT_OK = 0,
  PENT_EINVAL = -1,        /* invalid argument (host-side check, nothing launched) */
  PENT_ESINGULAR = -2,     /* a pivot alpha_i was zero or not finite (from pent_get_info) */
  PENT_ENOCONV = -3,       /* iterative refinement did not reach its tolerance (pent_get_info) */
  PENT_ECUDA = -4,         /* a CUDA runtime call failed */
  PENT_ENOTFACTORED = -5,  /* a solve was requested before any factorisation */
  PENT_ENOTBOUND = -6      /* the plan has no workspace/stream bound */
} pent_status;

typedef enum {
  PENT_F64 = 0,        /* FP64 factors, FP64 substitutions */
  PENT_F32_REFINE = 1  /* FP32 factors and substitutions, refined against an extended-precision residual */
} pent_precision;

/* Residual arithmetic used by PENT_F32_REFINE (pent_plan_set_option key PENT_OPT_RESIDUAL). */
typedef enum {
  PENT_RESIDUAL_FF = 0,   /* residual f - A x in double-FP32 ("float-float") arithmetic on the FP32 units */
  PENT_RESIDUAL_F64 = 1   /* residual f - A x in native FP64 */
} pent_residual;

typedef struct pent_plan pent_plan;

/*
 * Create a plan for `batch` independent systems.
 *   n_per_system: host array of `batch` row counts (each >= 1), or NULL when
 *                 every system has n_uniform rows.
 *   shared_matrix: nonzero when all systems share one matrix (the paper's
 *                 benchmark case, Sec. 3): the band/sigma arguments then
 *                 describe a single system and n_per_system must be NULL.
 *   precision:    PENT_F64 or PENT_F32_REFINE.
 *   tune_cache:   path of an autotuning cache (text, format below) or NULL for
 *                 the built-in choices.
 * The plan is a host object; it records shapes and choices only.
 * Errors: PENT_EINVAL for batch < 1, a row count < 1, shared_matrix with
 * uneven sizes, or a NULL `plan`; for PENT_F32_REFINE also a system longer
 * than 32,768 rows (one system is at most a cluster of 8 CTAs of 512
 * threads holding 8 rows each; PENT_F64 plans take any length).
 */
pent_status pent_plan_create(pent_plan** plan, int64_t batch, const int64_t* n_per_system, int64_t n_uniform,
                             int shared_matrix, pent_precision precision, const char* tune_cache);

/* Bytes of device workspace the plan needs (factors, scratch, info word). */
size_t pent_plan_workspace_bytes(const pent_plan* plan);

/*
 * Bind caller-owned device workspace (at least pent_plan_workspace_bytes,
 * 256-byte aligned) and a CUDA stream (cudaStream_t, may be NULL for the
 * legacy default stream).  Uploads the plan's small per-system tables with a
 * synchronous copy; this call is not capture-safe.  The workspace must stay
 * valid until the plan is destroyed or re-bound.
 */
pent_status pent_plan_bind(pent_plan* plan, void* d_workspace, void* cuda_stream);

/*
 * Autotuning cache.  A text file of rules, one per line; '#' starts a comment.
 *   f32 <n_lo> <n_hi> <rows_per_thread> <threads_per_system>
 *   f64 <n_lo> <n_hi> <unroll> <block_warps>
 * A PENT_F32_REFINE plan solves every system of n rows, n_lo <= n <= n_hi, with
 * the given CTA shape (rows per thread 4 or 8; threads per system as for
 * PENT_OPT_THREADS_PER_SYSTEM, their product covering n, or 0 for the fewest
 * threads that cover n with that many rows each).  A PENT_F64 plan
 * launches its groups of 32 systems (sorted by length) in runs of equal
 * settings, each group taking the rule of its longest system.  The first
 * matching rule of the plan's precision wins; systems no rule covers keep the
 * built-in choice.  pent_plan_create returns PENT_EINVAL for a cache that
 * cannot be read or has a malformed or impossible rule.  The cache is written
 * by the Python module paper_1807_07382_gb300.autotune, which times the
 * candidates on the GPU at hand.  Options set later with
 * pent_plan_set_option take precedence over the cache.
 *
 * Tuning options (keys below); values are integers.  Unknown keys or values
 * return PENT_EINVAL.  PENT_OPT_THREADS_PER_SYSTEM changes the factor layout
 * and the workspace size, so it is accepted only before pent_plan_bind (query
 * pent_plan_workspace_bytes after setting it).
 */
/* pent_solve_steps, pent_step_batch and adi_steps_2d keep the CUDA graphs they capture,
 * keyed by the field pointer, the step count and the settings, at most this many per plan;
 * beyond it the least recently launched graph is destroyed (one still running is freed
 * by the runtime when it completes) and a later call with its key captures it anew. */
#define PENT_MAX_CACHED_GRAPHS 16

enum {
  PENT_OPT_THREADS_PER_SYSTEM = 1, /* PENT_F64: 1 (one thread per system).  PENT_F32_REFINE: threads per
                                      system, 32 W with W <= 16 (one CTA) or 512 C with C <= 8 (a cluster of C
                                      CTAs); 8 rows per thread at most; 0 restores the automatic choice */
  PENT_OPT_RESIDUAL = 2,           /* pent_residual */
  PENT_OPT_BLOCK_WARPS = 3,        /* PENT_F64: warps per CTA of the solve kernels (1..8) */
  PENT_OPT_REFINE_TOL_LOG2 = 4,    /* refinement stops once the estimated remaining error, (max|dx| / max|x|)^2
                                      relative to max|x| after a step with correction dx, is <= 2^-tol (default 43) */
  PENT_OPT_UNROLL = 5,             /* PENT_F64: rows loaded ahead of the arithmetic: 2, 4 or 8 (default 4) */
  PENT_OPT_ROWS_PER_THREAD = 6,    /* PENT_F32_REFINE: rows per thread, 4 or 8, or 0 for the automatic choice
                                      (before pent_plan_bind, like PENT_OPT_THREADS_PER_SYSTEM) */
  PENT_OPT_PARTITION_ROWS = 7,     /* PENT_F64 per-system matrices: groups of 32 systems whose longest system
                                      has at least this many rows are solved in chunks of 256 rows joined by
                                      scans, instead of one serial walk per system; 0 never, -1 automatic
                                      (the default: where a walk would outlast the whole batch's streaming
                                      time, and at least 2048 rows).  Before pent_plan_bind. */
  PENT_OPT_PERIODIC = 8,           /* 1: the systems are cyclic (Sec. 2.3, Eq. matrix_sys1): row i reads
                                      x_{i-2} .. x_{i+2} with column indices modulo n, so the first two rows
                                      reach the last two columns and vice versa.  Plans of uniform n >= 5
                                      only, before pent_plan_bind.  PENT_F32_REFINE periodic plans take the
                                      periodic hyperdiffusion matrix (pent_factor_hyperdiff) and refine
                                      against the float-float residual; each FP32 solve is the solve of E
                                      followed by the 2 x 2 tail, with Z = E^{-1} k stored beside the
                                      factors (the matrix is symmetric, so h = k).  Solved by Navon's reduction as the
                                      paper describes it: the last two unknowns from a 2 x 2 system
                                      (Eq. first_two), the other n - 2 from the pentadiagonal E that remains
                                      (Eq. solve); everything that depends on the matrix alone (factors of E,
                                      E^{-T} h, L^{-1} k, the 2 x 2 inverse) is formed by the factorisation,
                                      so each solve is one forward and one back sweep.  pent_factor_batch takes
                                      the cyclic band; pent_factor_hyperdiff builds Eq. (matrix_sys) with
                                      sigma_x = sigma.  Adjoint, sigma-gradient and ADI calls return
                                      PENT_EINVAL for periodic plans. */
  PENT_OPT_CACHED_GRAPHS = 11,     /* read only (pent_plan_get_option): step graphs the plan holds now, at
                                      most PENT_MAX_CACHED_GRAPHS */
  PENT_OPT_FP32_KERNEL = 10,       /* PENT_F32_REFINE, not periodic: 0 (the default) solves with at most one
                                      refinement step and the float-float residual on the interior-constant
                                      kernel wherever the system's CTA shape allows it (one CTA of 1 to 16
                                      warps of 8 rows a thread, or one warp of 4): away from the walls
                                      the FP32 factors of I + sigma D4 settle on one pair of constants, which
                                      that kernel uses without loading them and whose chunk-map powers the
                                      factorisation stores; 1 solves every system with the general kernel that
                                      loads every row's factors.  Any time; results agree to the refinement's
                                      accuracy, not bit for bit. */
  PENT_OPT_CLUSTER_WARPS = 9,      /* PENT_F32_REFINE: systems that need more than 512 threads run in a
                                      thread-block cluster of up to 8 CTAs of exactly this many warps: 8
                                      (the default) or 4, which keep several CTAs resident per SM, or 16
                                      (CTAs of up to 16 warps, one per SM); systems longer than 8 such CTAs
                                      take the 16-warp form.  Systems of up to 512 threads run in one CTA
                                      whatever the value.  Before pent_plan_bind. */
  PENT_OPT_WINDOW_WARPS = 12,      /* PENT_F32_REFINE, not periodic: systems longer than R = 256 W rows (W
                                      this value: 4, the default, 8 or 16; 0 turns windows off) are solved,
                                      when a solve takes the interior-constant kernel, in windows of R rows,
                                      one CTA of W warps each, side by side in one launch.  A window starts
                                      and ends with zero states where it cuts the system and keeps only
                                      the rows at least O from a cut, O the overlap the factorisation finds
                                      per system: the fewest multiple of 8 rows over which both interior
                                      chunk maps of 8 rows shrink to 2^-56 (their powers bound how far a
                                      cut reaches: the rows kept equal the whole system's to far below
                                      FP64 rounding).  Systems whose overlap exceeds R / 8, or whose head
                                      of wall-dependent factors reaches the second window, keep their
                                      one-CTA or cluster shape.  Windows are laid out at factor time, which
                                      then reads the overlaps back and so waits for the plan's stream (a
                                      factorisation under a stream capture lays out none).  Before
                                      pent_plan_bind (the workspace reserves R / 8 overlap rows a side). */
  PENT_OPT_WINDOWS = 13,           /* read only: windows of the current factorisation (0: none; FP32 plans
                                      the PENT_OPT_WINDOW_WARPS windows, FP64 those of PENT_OPT_WINDOW_ROWS) */
  PENT_OPT_WINDOW_ROWS = 14,       /* PENT_F64, per-system matrices factored by pent_factor_hyperdiff: a
                                      group of 32 length-sorted systems whose padded length exceeds this
                                      many rows (1024, the default; a multiple of 64 in 256 .. 16384; 0
                                      turns windows off) is walked in windows of that many rows, all in
                                      one launch (PENT_OPT_WINDOW_FORM says how): a window enters each
                                      sweep with a zero state where it cuts a system and writes x only
                                      for the rows at least O from a cut, O the fewest multiple of 8 rows
                                      over which the interior row maps shrink to 2^-56.  The groups of a
                                      launch setting (a run of equal unroll, CTA width and partitioning)
                                      take windows only if each of their long groups has an overlap
                                      within 1/4 of the window (system windows; 1/8 for group windows);
                                      the others, and general bands (pent_factor_batch), keep their walks
                                      or partitioned solves.  The factorisation reads the overlaps back
                                      and so waits for the plan's stream (under a stream capture it lays
                                      out no windows).  Before pent_plan_bind (the workspace reserves
                                      the windows' room). */
  PENT_OPT_PERSISTENT = 15,        /* not periodic: 1 launches the windows (PENT_OPT_WINDOW_WARPS, and
                                      the group windows of PENT_OPT_WINDOW_ROWS) as a persistent grid, as many CTAs as stay
                                      resident, each taking windows in turn (bounded by the window count,
                                      no waits between CTAs); 0 (the default) one CTA (FP32) or warp (FP64)
                                      per window.  The same results either way. */
  PENT_OPT_FP64_INTERIOR = 16,     /* PENT_F64: 1 (the default) lets the walks of a hyperdiffusion
                                      factorisation (pent_factor_hyperdiff, per-system matrices) take the
                                      records of the interior rows from registers: rows 2 .. n - 3 of
                                      I + sigma D4 share one band row and the factorisation's row step
                                      settles, so past the first few dozen rows every row pair holds the
                                      same bits; the run of such pairs is found per system by
                                      pent_factor_hyperdiff (not by pent_refactor_solve_hyperdiff, after
                                      which the walks read every record until the next factorisation);
                                      0 reads every record from memory.  Bitwise the same results. */
  PENT_OPT_WINDOW_FORM = 17        /* PENT_F64, with PENT_OPT_WINDOW_ROWS: how the groups that take
                                      windows are walked.  1 (the default): system windows, one thread
                                      per window of one system, with that system's own overlap O (the
                                      fewest multiple of 8 rows over which its interior row maps shrink
                                      to 2^-56), listed in the order of the caller's rows so that a warp
                                      reads and writes neighbouring rows; every window but a system's
                                      last starts O rows before the first row not yet kept, the last
                                      ends at the system's end, and each walks window_rows rows (fewer
                                      for systems shorter than a window).  The forward and back walks
                                      are two launches, and the factorisation copies the windowed
                                      systems' records into a per-system layout (40 more workspace bytes
                                      a row of those systems: 1/alpha, beta/alpha, sigma/alpha, gamma,
                                      delta).  0: group windows, one warp per window of
                                      a group (all 32 systems cut at the same rows, the group's largest
                                      overlap).  Before pent_plan_bind (the workspace differs).  Both
                                      forms keep the rows at least O from every cut. */
};
pent_status pent_plan_set_option(pent_plan* plan, int key, int64_t value);
pent_status pent_plan_get_option(const pent_plan* plan, int key, int64_t* value);

/*
 * Host only: the windows (PENT_OPT_WINDOW_WARPS) of an n-row system cut into windows of
 * `window_rows` rows with `overlap` rows of overlap (both multiples of 8, 4 overlap <=
 * window_rows).  The first window covers rows [0, window_rows) and keeps [0, window_rows -
 * overlap); each next one starts `overlap` rows before the first row not yet kept and keeps
 * window_rows - 2 overlap rows; the last ends at row n and keeps the rest, so the kept rows
 * tile [0, n) once.  Writes, while `cap` lasts, four int32 per window into h_out4 (host memory,
 * may be NULL): first row, rows, then the first and the end of the kept rows relative to the
 * window; returns the number of windows, 0 when n <= window_rows (one CTA solves the system)
 * or the sizes do not qualify.
 */
int64_t pent_window_layout(int64_t n, int window_rows, int overlap, int32_t* h_out4, int64_t cap);

/*
 * Host only: the FP64 system windows (PENT_OPT_WINDOW_FORM 1) of an n-row system, windows of
 * `window_rows` rows with `overlap` rows of overlap (window_rows and overlap even, 0 < 4 overlap
 * <= window_rows; overlap 0 is allowed when n <= window_rows), in row pairs as the walks take
 * them.  A system of at most window_rows rows is one window; otherwise the first window covers
 * rows [0, window_rows) and keeps [0, window_rows - overlap), each next one starts `overlap` rows
 * before the first row not yet kept and keeps window_rows - 2 overlap rows, and the last covers
 * the window_rows rows (rounded up to a whole row pair) that end the system and keeps the rest,
 * so every window walks the same rows and the kept rows tile [0, n) once.  Writes, while `cap`
 * lasts, three int32 per window into h_out3 (host memory, may be NULL): the first row walked,
 * and the first and the end of the kept rows (absolute; the end clipped to n); returns the
 * number of windows, 0 for n <= 0 or sizes that do not qualify.
 */
int64_t pent_system_window_layout(int64_t n, int window_rows, int overlap, int32_t* h_out3, int64_t cap);

/*
 * The settings that solve system `system` (0 <= system < batch), as chosen by
 * options, the tune cache or the built-in rules: for PENT_F32_REFINE
 * *a = rows per thread and *b = threads per system; for PENT_F64 *a = unroll
 * and *b = warps per CTA of the launch that covers the system, or *a = 0 and
 * *b = rows per chunk when its group is solved by the partitioned kernels.
 */
pent_status pent_plan_system_config(const pent_plan* plan, int64_t system, int64_t* a, int64_t* b);

/*
 * Factor every system's band (Sec. 2.4, factorisation steps 1-14) into the
 * workspace.  a..e are device arrays of sum(n_s) doubles (n_0 doubles when the
 * matrix is shared), system-major.  Resets the info word.  A zero or
 * non-finite pivot is recorded (lowest system, its row) and reported by
 * pent_get_info as PENT_ESINGULAR; that system's solutions are unspecified.
 */
pent_status pent_factor_batch(pent_plan* plan, const double* a, const double* b, const double* c, const double* d,
                              const double* e);

/*
 * Build and factor A_s = I + sigma_s D4 for every system, where D4 is the
 * centred fourth difference of Sec. 2.2 (interior band [1, -4, 6, -4, 1]) on
 * a cell-centred grid with no-flux walls (ghost values mirror the cells next
 * to the wall, so D4 = D2N^2 with D2N the no-flux second difference).
 * d_sigma: device array of `batch` doubles (one when the matrix is shared),
 * each > 0.  The plan keeps sigma for the refinement residual.
 */
pent_status pent_factor_hyperdiff(pent_plan* plan, const double* d_sigma);

/*
 * x_s = A_s^{-1} f_s for every system (Sec. 2.4: L g = f, then R x = g).
 * f, x: device arrays of sum(n_s) doubles, system-major; x may alias f.
 * max_refine: PENT_F32_REFINE only -- at most this many refinement steps
 * (each: residual r = f - A x, correction A dx = r by the FP32 factors,
 * x += dx); 0 returns the plain FP32 solution.  Ignored for PENT_F64.
 */
pent_status pent_solve_batch(pent_plan* plan, const double* f, double* x, int max_refine);

/*
 * x_s = A_s^{-1} f_s for right-hand sides held in (pinned) host memory: h_f is
 * copied to the device staging array d_f, solved into d_x (as
 * pent_solve_batch; d_x may alias d_f) and copied back to h_x.  The batch is cut
 * into `nchunks` slices of whole systems that flow through three streams of
 * the plan -- copies in, solves, copies out, handed on slice by slice with
 * events -- so that the copy of one slice to the device, the solve of another
 * and the copy of a third back overlap (at most 256 slices; nchunks beyond
 * that, or beyond the number of systems, is clamped).  Slicing needs plans of one
 * system length solved by one launch shape (uniform batches, not periodic, no
 * partitioned groups); other plans run as one slice.  Asynchronous on the
 * plan's stream, which waits for every slice; h_f must stay unchanged and h_x
 * unread until the stream reaches that point.  Not capture-safe (host memory).
 *
 * Direct form (d_f = d_x = NULL, PENT_F32_REFINE plans): no staging and no
 * copies.  The FP32 solve kernels read each f row once from h_f and write each
 * x row once to h_x over the host link (NVLink-C2C on Grace-Blackwell nodes),
 * as pent_solve_batch would in device memory; h_x may alias h_f; nchunks is
 * ignored.  h_f and h_x must each lie, for all sum(n_s) doubles, inside one
 * page-locked allocation the device maps (cudaHostAlloc, pinned tensors); the
 * library checks this through the driver's pointer attributes before any
 * launch and returns PENT_EINVAL otherwise (pageable or device memory, a range
 * that runs past its allocation).  PENT_F64 plans: PENT_EINVAL (their
 * one-thread-per-system loads would cross the link 16 bytes at a time).
 */
pent_status pent_solve_host_batch(pent_plan* plan, const double* h_f, double* h_x, double* d_f, double* d_x,
                                  int nchunks, int max_refine);

/*
 * The check the direct form of pent_solve_host_batch makes on each of h_f and
 * h_x: PENT_OK when [h, h + bytes) lies inside one page-locked host allocation
 * that the device maps, PENT_EINVAL otherwise (NULL, bytes = 0, pageable or
 * device memory, a range past its allocation).  A host-side driver query: no
 * launch, no synchronisation, no plan needed.
 */
pent_status pent_host_range_mapped(const void* h, size_t bytes);

/*
 * `nsteps` implicit steps in place: x <- A^{-1} x, repeated.  The sequence is
 * captured once into a CUDA graph (keyed by x and nsteps) and replayed on
 * later calls; the factors stay resident.  The first call for a given key is
 * therefore not capture-safe; later calls are single graph launches.
 * PENT_F32_REFINE plans solved by the interior-constant kernel
 * (PENT_OPT_FP32_KERNEL 0, max_refine <= 1) keep each system's field in x as
 * a float pair per row (its high and low parts, scaled by a power of two held
 * in the workspace) between the steps of one call, so that only the first
 * step converts from FP64 and only the last back: x holds those pairs while
 * the call runs and FP64 values again once it has completed.
 */
pent_status pent_solve_steps(pent_plan* plan, double* x, int64_t nsteps, int max_refine);

/*
 * `nsteps` semi-implicit time steps in place on C (device, system-major), each
 *   A_s C^{k+1} = f,   f_i = C_i + mu_s (D2 (C^3 - C))_i - nu_s (D4 C)_i,
 * with f assembled inside the solve kernel from the old field (it is never
 * written to memory).  D2 and D4 are the centred second and fourth differences
 * of Sec. 2.2 on the plan's grid: periodic for PENT_OPT_PERIODIC plans, else
 * the cell-centred no-flux reflection of pent_factor_hyperdiff.  With
 * A_s = I + sigma_s D4:
 *   mu = D dt/dx^2, nu = 0, sigma = gamma D dt/dx^4: the semi-implicit
 *     Cahn-Hilliard step of Sec. 2.1 (Eq. temporal), one parameter set per
 *     system as in the parameter studies of Sec. 2.1;
 *   mu = 0, nu = sigma = dt/(2 dx^4): the Crank-Nicolson hyperdiffusion step of
 *     Sec. 2.2 (Eq. 1d_hyper_scheme).
 * d_mu, d_nu: device arrays of `batch` doubles (one when the matrix is
 * shared), or NULL for zero.  Several steps are captured once into a CUDA
 * graph (keyed by C, nsteps, d_mu, d_nu, max_refine) and replayed.  Plans:
 *   PENT_F64, periodic (any factorisation) or per-system no-flux factored by
 *     pent_factor_hyperdiff: f is assembled in FP64; max_refine is ignored;
 *   PENT_F32_REFINE (float-float residual), factored by pent_factor_hyperdiff:
 *     f is assembled in float-float arithmetic from C split into float pairs
 *     (no scaling: |C| must stay below 2^40, larger fields set the
 *     non-convergence flag), then solved in FP32 with up to max_refine
 *     refinement steps, as pent_solve_batch.
 * Other plans: PENT_EINVAL.
 */
pent_status pent_step_batch(pent_plan* plan, const double* d_mu, const double* d_nu, double* C, int64_t nsteps,
                            int max_refine);

/*
 * Re-assemble, re-factor and solve in one call: A_s = I + sigma_s D4 (as
 * pent_factor_hyperdiff) from a new d_sigma, then x_s = A_s^{-1} f_s.  This is
 * the paper's "Rewrite" use (Sec. 3), for matrices that change every step
 * (adaptive dt, varying coefficients).  For per-system matrices whose groups
 * are walked by one thread per system, the factorisation runs inside the
 * forward sweep of the same kernel; shared matrices and plans with
 * partitioned groups factor first and then solve.  The plan is left factored
 * with the new sigma (later pent_solve_batch calls reuse it); the info word is
 * reset.  f, x: as pent_solve_batch (x may alias f).  PENT_F64, non-periodic
 * plans only.
 */
pent_status pent_refactor_solve_hyperdiff(pent_plan* plan, const double* d_sigma, const double* f, double* x);

/*
 * Adjoint solve y_s = A_s^{-T} f_s from the stored factors: A^T = R^T L^T, so
 * R^T z = f (unit lower: z_i = f_i - gamma_{i-1} z_{i-1} - delta_{i-2} z_{i-2})
 * then L^T y = z (y_i = (z_i - beta_{i+1} y_{i+1} - epsilon_{i+2} y_{i+2}) /
 * alpha_i).  The transposed solve is not in the paper; it follows from its
 * factors (Sec. 2.4, the definitions of L and R).  Same layout and aliasing
 * rules as pent_solve_batch.  Matrices built by pent_factor_hyperdiff are
 * symmetric (A = I + sigma D2N^2), so for them A^{-T} f = A^{-1} f is computed
 * by the solve itself (either precision; max_refine as pent_solve_batch);
 * general bands need a PENT_F64 plan (others: PENT_EINVAL); periodic plans:
 * PENT_EINVAL.
 */
pent_status pent_adjoint_solve_batch(pent_plan* plan, const double* f, double* x, int max_refine);

/*
 * dL/dsigma_s contribution of one implicit step: g_sigma[s] -= mu_s . (D4 x_s)
 * for every system, with mu and x device arrays laid out like f (FP64
 * arithmetic, plans of either precision; periodic plans: PENT_EINVAL).  Used by
 * the differentiable time stepper (from A x^k = x^{k-1} and dA/dsigma = D4).
 */
pent_status pent_hyperdiff_sigma_grad(pent_plan* plan, const double* mu, const double* x, double* g_sigma);

/*
 * One alternating-direction step of the 2D Cahn-Hilliard equation on an
 * ny x nx grid with no-flux walls, in place on C (device, row-major, x fastest):
 *   rhs = mu L(C^3 - C) - sigma L(L C),  mu = dt/dx^2, sigma = gamma dt/dx^4,
 *   (I + sigma D4_x)(I + sigma D4_y) dC = rhs,  C <- C + dC - mean(dC).
 * L is the five-point Laplacian with the same wall reflection as D4.  The
 * paper names ADI for 2D problems without giving a scheme (Sec. 4); this is
 * the Douglas delta form of its semi-implicit step (Sec. 2.1).  Exact dC has
 * zero mean; removing the mean of the computed dC keeps the total mass to
 * rounding of C itself.
 * px: a PENT_F64 shared-matrix plan of ny systems of n = nx; it also holds
 *     the step's scratch (two fields and one accumulator).
 * py: a PENT_F64 shared-matrix plan of nx systems of n = ny.
 * Both must be bound to the same stream and factored by adi_plans_factor for
 * exactly this (gamma, dt, dx): the explicit part and the two sweeps then use
 * one sigma, and any other (gamma, dt, dx), or plans factored otherwise or
 * since, return PENT_EINVAL before anything is launched.  max_refine must be 0: the sweeps run
 * in FP64 (at sigma ~ 1e5 the FP32 factorisation would contract the error by
 * only ~0.2 per refinement step, and the field stays in L2, so there are no
 * HBM bytes for FP32 streaming to save).  Errors: PENT_EINVAL for mismatched
 * shapes, plans or parameters, PENT_ENOTFACTORED if either plan is not factored.
 */
pent_status adi_step_2d(pent_plan* px, pent_plan* py, double* C, int64_t nx, int64_t ny, double gamma, double dt,
                        double dx, int max_refine);

/*
 * Factor the two plans of an ADI step for (gamma, dt, dx): both take
 * A = I + sigma D4 with sigma = gamma dt / dx^4 (Sec. 2.1, the coefficient of
 * the implicit fourth-order term; D4 as in pent_factor_hyperdiff), computed
 * here once, and remember the three parameters for adi_step_2d / adi_steps_2d.
 * px, py as for adi_step_2d (shapes checked against each other: px has
 * py's n systems of py's batch rows).  Asynchronous and capture-safe (sigma
 * reaches the device as a kernel argument).  PENT_EINVAL for non-positive or
 * non-finite parameters or mismatched plans.
 */
pent_status adi_plans_factor(pent_plan* px, pent_plan* py, double gamma, double dt, double dx);

/* `nsteps` ADI steps, captured once into a CUDA graph and replayed. */
pent_status adi_steps_2d(pent_plan* px, pent_plan* py, double* C, int64_t nx, int64_t ny, double gamma, double dt,
                         double dx, int max_refine, int64_t nsteps);

/*
 * Synchronise the plan's stream and read the info word.  Returns PENT_OK,
 * PENT_ESINGULAR (bad_system/bad_row give the lowest failing system and its
 * row) or PENT_ENOCONV.  refine_steps_used: the largest number of refinement
 * steps any system needed since the last factorisation.  Output pointers may
 * be NULL.  Clears nothing.
 */
pent_status pent_get_info(pent_plan* plan, int64_t* bad_system, int64_t* bad_row, int* refine_steps_used);

/* Reset the info word (asynchronous, capture-safe). */
pent_status pent_clear_info(pent_plan* plan);

/*
 * Factor and solve `batch` systems of n rows each without allocating anything
 * (the paper has no counterpart to this entry point; it serves callers that
 * may not allocate device memory -- code that runs under a framework whose
 * allocator owns the GPU, plug-ins that are given buffers but no allocator, or
 * work that is about to be captured into a CUDA graph).  a..e, f, x: device
 * arrays of batch*n doubles, system-major as above; x may alias f.  d_info:
 * optional device word (may be NULL) that receives the lowest failing
 * (system << 32 | row) of a zero or non-finite pivot, or 0x7f7f7f7f7f7f7f7f.
 * Scratch: a fixed 32 MiB array owned by the library in every device's
 * memory, held from the moment a device loads the library until the process
 * exits; ceil(batch/32) * 32 * n * 24 bytes must fit in it (at most 1,344
 * systems of 1,024 rows: 42 warps of 32), otherwise PENT_EINVAL and nothing is
 * launched.  Every call whose stream is not being captured looks up the
 * array's device address in the current context; a call during a capture uses
 * the address an earlier call found in the same context, so make one call
 * before any stream capture (a capture without one returns PENT_ECUDA).  Every
 * call uses the same array, so
 * calls whose kernels may overlap on the GPU (unordered streams) race; order
 * them on one stream.  Asynchronous on cuda_stream; no cudaMalloc, cudaFree
 * or other allocating call is made.
 */
pent_status pent_gbsv_batch_noalloc(int64_t batch, int64_t n, const double* a, const double* b, const double* c,
                                    const double* d, const double* e, const double* f, double* x,
                                    unsigned long long* d_info, void* cuda_stream);

/*
 * Measurement probe (the paper has no counterpart): launch `blocks` CTAs of 256
 * threads, each thread running eight independent FP64 fused multiply-add
 * chains of 16 * iters steps, on cuda_stream (asynchronous).  *flops receives
 * the floating-point operations the launch performs (2 per FMA); time the
 * launch with events on the same stream to obtain the FP64 rate that bounds
 * the FP64 solves.  d_sink: one device double, written only in a case that
 * never occurs (it keeps the arithmetic from being removed).  PENT_EINVAL for
 * non-positive sizes or a misaligned or NULL pointer.
 */
pent_status pent_probe_fp64_fma(int64_t blocks, int64_t iters, double* d_sink, void* cuda_stream, double* flops);

/* Destroy a plan (host memory only; the workspace is the caller's). NULL is a no-op. */
void pent_plan_destroy(pent_plan* plan);

/* Static text for a status code. */
const char* pent_status_string(pent_status status);

/* Library version, e.g. "0.1.0". */
const char* pent_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PENTBATCH_H */
