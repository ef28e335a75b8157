/*
 * purify.h -- C-ABI of the GB300 SARA-SDMM imaging library (libpurify_gb300.so).
 *
 * The library solves the reweighted analysis problem of the paper's
 * Section 2.2, Eq. 3,
 *     min_{x in R_+^N} || W Psi^H x ||_1   subject to   || y - Phi x ||_2 <= eps,
 * by SDMM (Section 3, Algorithm 1) on one GPU, with SARA's reweighting as an
 * outer loop (Section 2.2).  It exposes the two operator pairs the method is
 * built from -- the measurement operator Phi (a Kaiser-Bessel NUFFT, Section 4)
 * with its adjoint, and the SARA dictionary Psi (Section 2.2) with its
 * adjoint -- and the solver.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: 0 (PURIFY_OK) on success, a negative purify_status otherwise.
 *   No entry point aborts the process.  purify_strerror() names a code.
 * - Pointers marked "device" are CUDA device pointers on the current device;
 *   the caller owns them and keeps them alive until the call has completed on
 *   `stream`.  The library never frees caller memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Operator calls are asynchronous on that stream; purify_sdmm_solve blocks
 *   until the solve has finished (its stats are then valid).
 * - Real arrays are float (precision PURIFY_FP32) or double (PURIFY_FP64),
 *   fixed when the operator is created.  Complex arrays are interleaved
 *   (re, im) pairs of that type.
 * - Images are n x n, row-major; pixel (i1, i2) sits at p = (i1 - n/2, i2 - n/2).
 *   Visibility m is y_m = sum_p x_p exp(-i (u_m p1 + v_m p2)) up to the
 *   NUFFT's approximation error (unnormalised; u pairs with rows).
 * - Visibility vectors passed across the ABI are in the caller's uv order;
 *   the library permutes internally.
 */
#ifndef PURIFY_H
#define PURIFY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct purify_op purify_op;

enum purify_precision { PURIFY_FP32 = 0, PURIFY_FP64 = 1 };

enum purify_status {
  PURIFY_OK = 0,
  PURIFY_ERR_INVALID = -1,       /* bad argument: null pointer, size, unsupported option */
  PURIFY_ERR_NOMEM = -2,         /* device allocation failed */
  PURIFY_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  PURIFY_ERR_TIMEOUT = -4,       /* a bounded device-side wait gave up */
  PURIFY_ERR_NOT_CONVERGED = -5, /* halting rule not met within t_max (x is still valid) */
  PURIFY_ERR_BUDGET = -6,        /* request exceeds the configured device-memory budget */
  PURIFY_ERR_CANCELLED = -7,     /* request cancelled by purify_server_cancel */
  PURIFY_ERR_NONFINITE = -8      /* the solve's objective or residual became NaN or infinite */
};

/*
 * purify_op_create -- build the measurement operator Phi = G F Z S for a
 * fixed uv coverage (Section 4: a non-uniform FFT from the discrete image to
 * continuous visibilities) and the SARA dictionary for `dwt_levels` levels.
 *   uv          device, double[M][2]: (u_m, v_m) in radians per pixel, any
 *               real values (taken modulo 2 pi onto [-pi, pi)).
 *   M           number of visibilities, 1 <= M < 2^31.
 *   n           image side; a power of two, 16 <= n <= 2048.
 *   oversample  grid oversampling alpha; must be 2 (grid side K = 2n).
 *   J           Kaiser-Bessel support in grid cells; must be 8.
 *   dwt_levels  wavelet levels L, 1 <= L, with n / 2^L >= 2.
 *   precision   PURIFY_FP32 (float storage, FP64 reductions) or PURIFY_FP64.
 *   stream      stream for the set-up kernels (uv binning, tables).
 *   out         receives the new operator; untouched on error.
 * PURIFY_ERR_INVALID (purify_last_error says which) for a non-finite uv.
 * The operator owns device copies of the sorted uv tiles and tables and is
 * released by purify_op_destroy.  Synchronises `stream` before returning.
 * Set-up temporaries (binning scratch; later, the PSF operator of the
 * convolution form) come from a per-device memory pool of the library that
 * keeps up to 1 GiB of released memory mapped for the next creation.
 */
int purify_op_create(const double* uv, int64_t M, int n, int oversample, int J,
                     int dwt_levels, int precision, void* stream, purify_op** out);

/* Work decomposition of the gridding kernels (0 = default). */
typedef struct {
  int tile;   /* uv tile side in grid cells: 8 (default) or 16 */
  int chunk;  /* visibilities per work item, 64..8192 (default by M: 256 below 2^20,
                 2048 from 2^21, 1024 between -- the autotuner's usual choices) */
} purify_op_options;

/* purify_op_create_ex -- purify_op_create with an explicit tile / chunk. */
int purify_op_create_ex(const double* uv, int64_t M, int n, int oversample, int J, int dwt_levels,
                        int precision, const purify_op_options* opt, void* stream, purify_op** out);

/*
 * purify_autotune -- time Phi + Phi^H as the solver applies them (visibilities
 * in the operator's sorted order; `reps` pairs after one warm-up) for every
 * tile in {8, 16} and chunk in {256, 512, 1024, 2048} on this uv coverage and
 * return the fastest options (and their time per pair in ms); candidates
 * within 2% of the fastest count as ties, won by the largest chunk.
 * Builds and frees one operator per candidate; synchronises `stream`.
 */
int purify_autotune(const double* uv, int64_t M, int n, int dwt_levels, int precision, int reps,
                    void* stream, purify_op_options* best, double* best_ms);

/* purify_op_destroy -- free everything the operator owns (NULL is a no-op). */
int purify_op_destroy(purify_op* op);

/*
 * purify_op_info -- report sizes fixed at creation (any pointer may be NULL):
 * image side, visibility count, grid side K, uv tile side, work items,
 * precision, and device bytes owned by the operator.
 */
int purify_op_info(const purify_op* op, int* n, int64_t* M, int* K, int* tile,
                   int* n_items, int* precision, int64_t* device_bytes);

/*
 * purify_phi -- y = Phi x (Section 4 NUFFT: deapodise S, zero-pad Z,
 * 2D FFT F, Kaiser-Bessel degridding G).
 *   x  device, real[n][n];   y  device, complex[M] (caller's uv order).
 */
int purify_phi(purify_op* op, const void* x, void* y, void* stream);

/*
 * purify_phi_adj -- x = Re(Phi^H y): gridding G^H, inverse FFT, crop Z^T and
 * deapodise S.  This is the adjoint of Phi restricted to real images (the
 * problem is posed on R_+^N, Eq. 2-3), so <Phi x, y> = <x, Phi^H y> in the
 * real inner product.
 *   y  device, complex[M] (caller's uv order);   x  device, real[n][n].
 */
int purify_phi_adj(purify_op* op, const void* y, void* x, void* stream);

/*
 * purify_sara_fwd -- c = Psi^H x (Section 2.2): the Dirac basis and the
 * Daubechies Db1..Db8 periodic orthonormal wavelet bases with `dwt_levels`
 * levels, each scaled by 1/sqrt(9) so that Psi Psi^H = I -- or the q bases
 * selected by purify_op_set_dictionary, each scaled by 1/sqrt(q).
 *   x  device, real[n][n];   c  device, real[q][n][n] (q = 9 by default),
 *   basis-major in increasing basis order (Dirac first, then Db_K in Mallat
 *   layout).
 */
int purify_sara_fwd(purify_op* op, const void* x, void* c, void* stream);

/* purify_sara_adj -- x = Psi c, the adjoint (and left inverse) of purify_sara_fwd. */
int purify_sara_adj(purify_op* op, const void* c, void* x, void* stream);

/*
 * purify_sara_fwd_static -- the same c = Psi^H x as purify_sara_fwd (FP32),
 * for callers that cannot allocate device memory: no operator is needed and
 * the call makes no cudaMalloc, cudaFree or other allocating call.  (The
 * paper has no counterpart; this serves pipelines that reserve all device
 * memory up front and must not allocate while streaming, or hosts that hand
 * the library pre-sized buffers only.)
 *   x  device, float[n][n];  c  device, float[9][n][n] (as purify_sara_fwd).
 *   n  a power of two, 16 <= n <= 512; n / 2^levels >= 2.  Larger n returns
 *      PURIFY_ERR_INVALID (purify_last_error names the limit).
 * The multi-level scratch lives in one fixed 4 MiB device array per device,
 * held until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current;
 * with CUDA's lazy module loading that lookup is also what loads this
 * function's device code and so reserves the 4 MiB: make the first call at
 * start-up, where that one reservation is acceptable, and before any stream
 * capture.  Later calls reserve nothing.  Every call shares the array, which
 * keeps the last call's contents (each call overwrites what it reads, so
 * nothing needs clearing): calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  A launch error
 * is reported through cudaPeekAtLastError, which leaves the error state as
 * it was (an error pending from earlier work is reported too).
 */
int purify_sara_fwd_static(const float* x, float* c, int n, int levels, void* stream);

/*
 * purify_op_set_dictionary -- choose the sparsity dictionary Psi of the
 * operator's analysis calls and of purify_sdmm_solve's l1 block (Section 4
 * compares the same problem under other dictionaries: BP is the Dirac basis
 * alone, BPDb8 the Db8 basis alone, BPSA all nine bases without reweighting;
 * with n_reweight > 0 the solve is the reweighted RWBP / RWBPDb8 / SARA).
 *   mask  bit 0 the Dirac basis, bit K (1..8) the Daubechies DbK basis; the
 *         q selected bases are each scaled by 1/sqrt(q) (Psi Psi^H = I).
 *         The default is 0x1FF (SARA).
 * PURIFY_ERR_INVALID for mask 0, bits above 8, or while a resumable solve is
 * active on the operator.  purify_op_dictionary returns the mask and q.
 */
int purify_op_set_dictionary(purify_op* op, unsigned mask);
int purify_op_dictionary(const purify_op* op, unsigned* mask, int* n_bases);

/*
 * purify_op_set_prior -- the prior of purify_sdmm_solve's first block.
 * Section 4 solves the same constrained problem with total variation in
 * place of the l1 analysis prior ("TV"; with n_reweight > 0 the reweighted
 * "RWTV").
 *   prior 0: ||W Psi^H x||_1 over the dictionary of purify_op_set_dictionary
 *            (the default; SARA and its sub-dictionaries).
 *   prior 1: TV_W(x) = sum_ij w_ij |(grad x)_ij|, the weighted isotropic total
 *            variation with forward differences and a zero difference past the
 *            last row and column; L_1 = I, so the composite operator is still
 *            Phi^H Phi + 2I.  Its proximity operator (Eq. 7) is computed on
 *            the dual: prox(v) = v + div q, q from `tv_iters` projected-gradient
 *            steps q <- P(q + (1/8) grad(v + div q)) onto |q_ij| <= gamma w_ij,
 *            warm-started from the previous SDMM iteration's q (zero at the
 *            start of every round).  RWTV weights w_i = delta / (delta +
 *            |grad x_hat|_i), delta from the same schedule as SARA's applied
 *            to the gradient magnitudes.  The default gamma is
 *            1e-3 ||nu^2 Re Phi^H y||_inf; the objective reported is TV_W.
 *   tv_iters 1..100000 (prior 1; ignored for prior 0).
 * PURIFY_ERR_INVALID for other values or while a resumable solve is active.
 */
int purify_op_set_prior(purify_op* op, int prior, int tv_iters);

/*
 * purify_op_set_blocks -- partition the visibilities into R blocks (Eq. 4):
 * the solver then imposes one constraint ||y_b - Phi_b x||_2 <= eps_b per
 * block (Eq. 5), i.e. S = R + 2 functions in Eq. 6, each block with its own
 * l2-ball projection; the composite operator sum_b Phi_b^H Phi_b = Phi^H Phi is
 * unchanged (Section 3).  Visibilities are re-binned by (block, uv tile).
 *   block_ids  device, int32[M] in the caller's uv order, values in [0, R);
 *              may be NULL when R == 1 (one block).
 *   R          1 <= R <= 64.
 * Synchronises `stream`; PURIFY_ERR_INVALID for out-of-range ids.
 */
int purify_op_set_blocks(purify_op* op, const int* block_ids, int R, void* stream);

/*
 * purify_gram -- out = Re(Phi^H Phi x), the data term of the composite
 * operator sum_i L_i^H L_i = Phi^H Phi + 2I that the SDMM global update
 * inverts (Section 3).
 *   mode 0: Phi then Phi^H through the NUFFT (degridding and gridding fused).
 *   mode 1: the composite precomputed once, as Section 3 suggests: the PSF
 *           k(d) = sum_m exp(i (u_m d1 + v_m d2)) over offsets d in [-n, n)^2
 *           (from the NUFFT adjoint of unit visibilities on a 2n x 2n image)
 *           applied as a circular convolution on the 2n grid; needs n <= 1024.
 *           It equals the exact (NUDFT) normal operator up to the NUFFT error
 *           of the PSF.  The first call builds and keeps the real half
 *           spectrum ((K/2 + 1) K reals of operator memory; its set-up
 *           buffers come from the set-up pool; synchronises `stream`).
 *   x, out  device, real[n][n].
 */
int purify_gram(purify_op* op, const void* x, void* out, int mode, void* stream);

/* Solver parameters (Algorithm 1 and the SARA loop). */
typedef struct {
  double eps;         /* l2 bound on the noise, Eq. 2-3 (> 0) */
  double gamma;       /* SDMM step gamma > 0; <= 0 selects 1e-3 ||Psi^H (nu^2 Phi^H y)||_inf */
  double nu;          /* scale applied to Phi inside SDMM (problem unchanged); <= 0 selects 1/||Phi||_2 */
  int t_max;          /* SDMM iterations per reweighting round (>= 1) */
  int cg_iters;       /* conjugate-gradient steps per global update (>= 1) */
  double xi;          /* relative objective change for halting; 0 runs exactly t_max iterations */
  int n_reweight;     /* reweighted solves after the first, unweighted one (>= 0) */
  double delta0;      /* first reweighting delta; <= 0 selects std of the round-0 coefficients */
  double delta_min;   /* lower bound on delta; <= 0 selects 1e-4 * delta_1 */
  double delta_decay; /* delta_k = max(decay^(k-1) delta_1, delta_min); <= 0 selects 0.1 */
  int warm_start;     /* non-zero: each reweighted round starts from the previous solution */
  int power_iters;    /* power-iteration steps used when nu <= 0 (>= 1) */
  int use_graph;      /* non-zero: replay one SDMM iteration as a captured CUDA graph (the operator
                         keeps it for later solves with the same nu, gamma, eps, cg_iters,
                         dictionary, prior and blocks) */
  int gram;           /* CG operator Re(Phi^H Phi): 0 NUFFT (G^H G each application), 1 precomputed
                         composite as a PSF convolution (Section 3), -1 the latter when n <= 1024 */
  const double* eps_blocks; /* host, one bound per visibility block (Eq. 5) when
                               purify_op_set_blocks gave R > 1; NULL: eps sqrt(M_b / M) */
} purify_params;

/* Solver statistics, filled by purify_sdmm_solve. */
typedef struct {
  int iterations;       /* SDMM iterations run, all rounds */
  int rounds;           /* SARA rounds run (1 + reweighted) */
  int converged;        /* halting rule met in the last round (always 0 when xi == 0) */
  double objective;     /* ||W Psi^H x||_1 at the returned x, last round's W */
  double residual;      /* ||y - Phi x||_2 at the returned x (all blocks) */
  double nu;            /* scale used for Phi inside SDMM */
  double gamma;         /* gamma used */
  double elapsed_ms;    /* wall time of the solve on the device stream */
} purify_stats;

/*
 * purify_sdmm_solve -- SARA: solve Eq. 3 with W = I by SDMM (Algorithm 1),
 * then `n_reweight` times update W from the last solution and solve again.
 *   y      device, complex[M], caller's uv order (the measured visibilities).
 *   params host, read only.
 *   x_out  device, real[n][n]: the last round's x_hat.
 *   stats  host, may be NULL.
 * Blocks until the solve has finished on `stream`.  Returns
 * PURIFY_ERR_NOT_CONVERGED (with a valid x_out) when xi > 0 and the halting
 * rule was not met within t_max in the last round; PURIFY_ERR_INVALID for a
 * y holding NaN or infinity (checked once at the start); PURIFY_ERR_NONFINITE
 * when the final objective or residual is not finite; PURIFY_ERR_TIMEOUT
 * when a bounded device wait gave up.
 */
int purify_sdmm_solve(purify_op* op, const void* y, const purify_params* params,
                      void* x_out, purify_stats* stats, void* stream);

/*
 * purify_batch_solve -- many independent SARA solves (Eq. 3 by Algorithm 1,
 * as purify_sdmm_solve; e.g. frequency channels or fields) advanced
 * together.  Instances are grouped by image side; within a group every pass
 * of an SDMM iteration (CG passes, degridding, gridding, projections, SARA
 * levels, vector steps) is one kernel launch over all of the group's
 * instances, reading each instance's arguments from a device table, and one
 * SDMM iteration of the whole batch is one captured CUDA graph in which the
 * groups run side by side.
 *   count   number of instances (>= 1).
 *   ops     count distinct operators of one precision, image sides 64..1024,
 *           one visibility block, the l1 prior (any dictionary).
 *   y       count device pointers, each instance's visibilities (caller order).
 *   params  count parameter sets: each instance's eps, gamma, nu (<= 0:
 *           computed per instance as in purify_sdmm_solve), delta rules; t_max,
 *           cg_iters and n_reweight equal for all, xi = 0 (fixed counts); the
 *           CG operator is the precomputed convolution form (gram 0 refused).
 *   x_out   count device pointers, real[n_i][n_i].
 *   stats   host, count entries, may be NULL.
 * Each instance's result equals its purify_sdmm_solve up to rounding (the
 * gridding atomics and the order of partial sums).  Blocks until done;
 * PURIFY_ERR_INVALID (purify_last_error says which rule) for instances the
 * batch cannot group.
 */
int purify_batch_solve(int count, purify_op* const* ops, const void* const* y, const purify_params* params,
                       void* const* x_out, purify_stats* stats, void* stream);

/*
 * Resumable solve and checkpoints.  purify_sdmm_solve is begin + steps + end
 * in one call; the three parts are also public so that a caller can stop
 * between SDMM iterations, save the solver state to host memory, and resume
 * it later -- in this process or another -- on an operator built from the
 * same uv coverage, image side, levels, precision, dictionary and blocks.
 *
 * purify_solve_begin -- check y, take nu and gamma (computed as in
 *   purify_sdmm_solve when <= 0), set up round 0; y and params as for
 *   purify_sdmm_solve (params copied; y read before the call returns).
 * purify_solve_step -- run up to max_iters SDMM iterations (Algorithm 1 steps
 *   5-10, rounds advancing as in the SARA loop), then wait for them; *done is
 *   set to 1 once the last round has finished.  Returns PURIFY_ERR_TIMEOUT if
 *   a bounded device wait gave up.
 * purify_solve_end -- copy the last x_hat to x_out (device real[n][n]), fill
 *   stats, release the solve; statuses as purify_sdmm_solve.
 * purify_solve_state_bytes -- size of a checkpoint of this operator's solve.
 * purify_solve_save -- write the state after the last completed iteration to
 *   `host` (bytes >= purify_solve_state_bytes): a header (format version,
 *   precision, n, M, dictionary size, blocks, round, iteration counters,
 *   convergence state, nu, gamma, the first reweighting delta, the last
 *   objective) followed by x_hat, sum_i x_i, z_1, z_2, the SARA weights W and
 *   z_3 (reals of the operator's precision; z_3 in the operator's sorted
 *   visibility order).  CG vectors are not state: every SDMM iteration
 *   restarts its CG from x_hat.
 * purify_solve_load -- after purify_solve_begin with the same y and
 *   parameters, replace the fresh state by a saved one; the next
 *   purify_solve_step continues where the saved solve stopped.
 *   PURIFY_ERR_INVALID when the checkpoint does not match the operator.
 * The resumed solve runs the same kernels in the same order; gridding sums
 * with atomics, so a resumed and an uninterrupted solve agree to rounding,
 * not bit for bit.
 */
int purify_solve_begin(purify_op* op, const void* y, const purify_params* params, void* stream);
int purify_solve_step(purify_op* op, int max_iters, int* done);
int purify_solve_end(purify_op* op, void* x_out, purify_stats* stats, void* stream);
int purify_solve_state_bytes(const purify_op* op, int64_t* bytes);
int purify_solve_save(purify_op* op, void* host, int64_t bytes);
int purify_solve_load(purify_op* op, const void* host, int64_t bytes);

/*
 * Failure detection (the paper has no counterpart).  Every mbarrier wait of
 * the library's kernels (TMA patch loads in degridding, bulk operand copies
 * in the CG row passes) is bounded: after its budget of try-wait spins it
 * raises a device error flag, lets any copy still in flight land (a second,
 * fixed budget), skips its work and returns, and the next synchronising call
 * reports PURIFY_ERR_TIMEOUT; the context stays usable.
 * purify_set_wait_limit -- set the first-phase budget (spins; 0 restores the
 *   default 2^24) on the current device, for tests and diagnostics.
 * purify_wait_selftest -- one CTA arms an mbarrier for 16 bytes and, with
 *   deliver != 0, brings them by a bulk copy (returns PURIFY_OK); with
 *   deliver == 0 nothing is ever sent, the wait runs out of its budget and
 *   the call returns PURIFY_ERR_TIMEOUT.  Blocks on `stream`.
 */
int purify_set_wait_limit(uint32_t spins);
int purify_wait_selftest(int deliver, void* stream);

/*
 * Kernel timing (instrumentation; the paper has no counterpart).  While
 * enabled, every kernel the operator launches is bracketed by CUDA events on
 * its stream and the solver runs without graph replay; purify_profile_read
 * returns, per kernel kind, the summed device time and launch count since
 * profiling was enabled.  Kinds: 0 row_fwd, 1 col_fwd, 2 degrid, 3 grid,
 * 4 gram, 5 col_inv, 6 row_inv, 7 sara_analysis, 8 sara_synthesis,
 * 9 vector (CG updates and scalar finalisation), 10 memset, 11 col_conv,
 * 12 row_fwd_h, 13 row_inv_h (the row passes of the convolution form),
 * 14 tv (the TV block of purify_op_set_prior).
 */
enum { PURIFY_NUM_KERNEL_KINDS = 15 };
int purify_profile(purify_op* op, int enable);
int purify_profile_read(purify_op* op, int kind, double* total_ms, int64_t* launches);
const char* purify_kernel_name(int kind);

/*
 * Request server (continuous batching; the paper has no counterpart -- it is
 * the serving form of Algorithm 1 for many independent imaging requests).
 * Requests wait in a FIFO queue; each scheduling pass admits queued requests
 * while a slot is free and their estimated device memory
 * (purify_estimate_bytes) fits the budget, and keeps each admitted solve's
 * image, dual variables and sorted uv tiles resident on the device.  Every
 * admitted solve runs one SDMM iteration at a time on its own stream, so
 * that the solves' kernels overlap; a solve whose iteration has completed
 * gets its halting test and its next iteration in the next pass, while one
 * still running is left alone (no lock-step: a large image never holds back
 * a small one).  A finished solve frees its slot and memory at once.
 * Iteration-level batching (off by default, purify_server_set_batching): admitted solves that share
 * image side, precision, CG steps and dictionary, use the convolution form of
 * the CG operator (64 <= n <= 1024) and one visibility block advance together
 * -- one SDMM iteration of all of them is one batched graph, each pass one
 * launch over the group as in purify_batch_solve, cached while the group's
 * membership is unchanged; a ready solve whose group is in flight joins it at
 * the next iteration.  The
 * device memory of admitted solves comes from a stream-ordered memory pool
 * of the server that keeps up to `budget_bytes` mapped, so admitting and
 * releasing solves never synchronises the device; host inputs are staged
 * through pinned memory on the server's own stream.  The caller drives the
 * server with purify_server_step; not thread-safe.  All solves run on the
 * current device (at create time).
 */
typedef struct purify_server purify_server;
int purify_server_create(int64_t budget_bytes, int max_slots, purify_server** out);
int purify_server_destroy(purify_server* srv);
/* Work decomposition used for requests of image side n (e.g. from purify_autotune). */
int purify_server_set_options(purify_server* srv, int n, const purify_op_options* opt);
/* Copies uv (host double[M][2]) and y (host complex[M] of the precision) and
 * queues the request; PURIFY_ERR_BUDGET if it can never fit the budget;
 * PURIFY_ERR_INVALID (purify_last_error names the array and visibility) if
 * uv or y holds NaN or infinity -- nothing is queued then. */
int purify_server_submit(purify_server* srv, const double* uv_host, const void* y_host, int64_t M, int n,
                         int dwt_levels, int precision, const purify_params* params, int* request_id);
/* One scheduling pass; reports how many solves are active and queued after it. */
int purify_server_step(purify_server* srv, int* n_active, int* n_queued);
/* Iteration-level batching on (enable != 0) or off (0, the default). */
int purify_server_set_batching(purify_server* srv, int enable);
/* Solve-iterations launched so far in batched groups and on their own. */
int purify_server_counts(purify_server* srv, int64_t* batched, int64_t* solo);
/* Cancel a queued or running request: a queued one leaves the queue; a
 * running one is stopped between SDMM iterations (the call waits for the
 * iteration in flight on that solve's stream only) and its memory and slot
 * are released.  Its result is PURIFY_ERR_CANCELLED afterwards.
 * PURIFY_ERR_INVALID for an unknown or already finished request. */
int purify_server_cancel(purify_server* srv, int request_id);
/* 1 and the image (host real[n][n]), stats, latency (submit to done) and
 * queueing time (submit to admission) when the request has finished; 0 while
 * it is queued or running; its negative status if it failed. */
int purify_server_result(purify_server* srv, int request_id, void* x_host, purify_stats* stats,
                         double* latency_s, double* queue_s);
/* Device bytes an operator plus solver state of this size may hold (an upper
 * bound used for admission, including the transient PSF set-up). */
int purify_estimate_bytes(int64_t M, int n, int dwt_levels, int precision, int64_t* bytes);

/* purify_default_params -- the defaults described in purify_params. */
void purify_default_params(purify_params* p);

/* purify_strerror -- static description of a status code. */
const char* purify_strerror(int status);

/* purify_last_error -- detail of the calling thread's last failure (which
 * call, where, the CUDA error name); empty if none.  Valid until the next
 * failing call on this thread. */
const char* purify_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PURIFY_H */
