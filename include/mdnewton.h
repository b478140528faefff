/*
 * mdnewton.h -- C-ABI of libmdnewton: Newton's method on truncated power
 * series in multiple double arithmetic on one GB300 GPU (sm_103a).
 *
 * Method (J. Verschelde, "GPU Accelerated Newton for Taylor Series Solutions
 * of Polynomial Homotopies in Multiple Double Precision", arXiv 2301.12659):
 * one Newton step evaluates and differentiates a polynomial system f at a
 * vector of truncated power series x(t) (Section 5.1: forward, backward and
 * cross products of every monomial), then solves the block lower triangular
 * Toeplitz system A(t) dx(t) = -f(x(t)) mod t^(d+1) (Section 2, Eq.
 * (eqToeplitz)) with a Householder QR of the leading matrix A0 (Section 5.3)
 * and forward substitution dx_k = A0^{-1} (b_k - sum_{j>=1} A_j dx_{k-j}),
 * and updates x := x + dx.  The calls follow the problem statement of
 * Section 2 (input: the system with series coefficients, the leading
 * coefficients of the start series, the number of iterations; output: the
 * series and the residuals).
 *
 * Numbers.  A multiple double (md) with K limbs (K = 2 double double, 4 quad
 * double, 8 octo double) is an unevaluated sum of K nonoverlapping doubles
 * (Section 1.2).  Complex data (C = 2) have a real and an imaginary md part.
 *
 * Layout.  Every md array is structure of arrays, one array per limb and part
 * (Section 1.2): an array of N md values is float64 [K][C][N], element
 * (limb l, part c, index i) at offset (l*C + c)*N + i.  Concretely
 *   series    x, f, dx   [K][C][n][d+1]    coefficient k of variable v at i = v*(d+1) + k
 *   coeffs    coeff      [K][C][M][d+1]    coefficient k of monomial m at i = m*(d+1) + k
 *   Jacobian  A          [K][C][d+1][n][n] entry (j, i, v) at i' = (j*n + i)*n + v
 * where A_j[i][v] = [t^j] d f_i / d x_v.
 *
 * System.  Equation i is f_i = sum_{m : eq[m] = i} coeff_m(t) prod_{p} x_{var_idx[p]}(t)
 * + cst_i(t), the product over p = var_ptr[m] .. var_ptr[m+1]-1 (a repeated
 * variable index is a power).  Linear terms such as a diagonal 64 x_i are
 * monomials with one variable and a constant coefficient series.
 *
 * Ownership.  The library allocates no device memory.  The caller allocates
 * every device buffer, including the workspace sized by
 * mdn_workspace_bytes(); the library borrows the pointers until the next
 * mdn_load_system() or mdn_destroy().  All device work is enqueued on the
 * stream given to mdn_load_system().  Host pointers are only read during the
 * call.
 *
 * Errors.  Every call returns an mdn_status and never throws.  Device-side
 * conditions (zero pivot in the QR of A0, non-finite values, a bounded wait
 * that timed out) are collected in a status word and reported by the call
 * that synchronises (mdn_newton, mdn_solve, mdn_status_word).
 * mdn_last_error() gives a message for the last failure on a context.
 */
#ifndef MDNEWTON_H
#define MDNEWTON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdn_ctx mdn_ctx;

typedef enum {
  MDN_OK = 0,
  MDN_EINVAL = 1,          /* invalid argument or size */
  MDN_ECUDA = 2,           /* a CUDA runtime call failed */
  MDN_ESINGULAR = 3,       /* A0 has a zero pivot (Householder norm 0) */
  MDN_ENONFINITE = 4,      /* a non-finite value appeared in the series */
  MDN_ENOTCONVERGED = 5,   /* tolerance not met within max_steps; x readable */
  MDN_ETIMEOUT = 6,        /* a bounded device wait gave up */
  MDN_ESTATE = 7,          /* call out of order (no system or series loaded) */
  MDN_EWORKSPACE = 8,      /* workspace smaller than mdn_workspace_bytes() */
  MDN_ETOOLARGE = 9        /* sizes beyond MDN_STATIC_SCRATCH_BYTES (mdn_evaluate_static) */
} mdn_status;

/* Most Newton steps one mdn_newton() call may run (size of the device history). */
#define MDN_MAX_STEPS 64
/* Largest truncation degree supported (d+1 <= 64 coefficients). */
#define MDN_MAX_DEGREE 63
/* Largest number of equations and unknowns of a context that solves.  Up to
 * MDN_MAX_N_DATAFLOW the QR of A0 is one cooperative dataflow launch that
 * keeps its columns and rows in shared memory (a warp per column of A0 and
 * of the identity, a warp per two rows of R^{-1}; all 5n/8 blocks resident,
 * one per SM); above it the QR runs column by column with the columns in
 * global memory (three launches per reflector, the paper's n = 1024
 * workloads). */
#define MDN_MAX_N 1024
#define MDN_MAX_N_DATAFLOW 192
/* Largest n of a context that only evaluates (mdn_evaluate, mdn_get_residual;
 * mdn_newton, mdn_solve and mdn_adjoint return MDN_EINVAL above MDN_MAX_N). */
#define MDN_MAX_N_EVAL 4096

/* Create a context for K limbs (2, 4 or 8; 1 runs plain doubles), real
 * (is_complex = 0) or complex (1) data, 1 <= n <= MDN_MAX_N equations and
 * unknowns (up to MDN_MAX_N_EVAL for a context that only evaluates) and
 * truncation degree 0 <= degree <= MDN_MAX_DEGREE.  *out receives the context
 * (host memory); MDN_EINVAL on bad sizes, MDN_ECUDA without a usable GPU. */
mdn_status mdn_create(mdn_ctx** out, int limbs, int is_complex, int n, int degree);

/* Bytes of device workspace mdn_load_system() needs for a system of
 * n_monomials monomials with CSR offsets var_ptr (host, n_monomials+1
 * entries).  Returns 0 on invalid arguments. */
size_t mdn_workspace_bytes(const mdn_ctx* ctx, int n_monomials, const int32_t* var_ptr);

/* Load the system (Section 2 problem statement: f with power series
 * coefficients and the truncation degree d).
 *   eq_of_monomial [M]    host, equation of each monomial (0 <= eq < n)
 *   var_ptr       [M+1]   host, CSR offsets into var_idx, var_ptr[0] = 0,
 *                         at least one variable per monomial
 *   var_idx       [nnz]   host, variable indices (0 <= v < n)
 *   coeff         device, [K][C][M][d+1]
 *   const_term    device, [K][C][n][d+1]
 *   workspace     device, >= mdn_workspace_bytes() bytes, 256-byte aligned
 *   cuda_stream   a cudaStream_t (NULL = legacy default stream)
 * The call copies the structure into the workspace and synchronises the
 * stream once.  coeff and const_term are read by later calls, not copied. */
mdn_status mdn_load_system(mdn_ctx* ctx, int n_monomials, const int32_t* eq_of_monomial,
                           const int32_t* var_ptr, const int32_t* var_idx, const double* coeff,
                           const double* const_term, void* workspace, size_t ws_bytes,
                           void* cuda_stream);

/* Set the current series x(t) (device [K][C][n][d+1], copied on the stream). */
mdn_status mdn_set_series(mdn_ctx* ctx, const double* x);

/* Run Newton steps (Section 2 pseudo code) from the current series.  With
 * tol <= 0 exactly max_steps steps run with one synchronisation at the end;
 * with tol > 0 the loop stops after the first step whose ||dx||_1 <= tol
 * (MDN_ENOTCONVERGED if none).  steps_done (host, may be NULL) receives the
 * number of steps run; res_hist (host, may be NULL) receives per step the
 * three doubles ||f(x)||_1 before the update, the residual
 * ||b - A dx||_1 of the linear solve (b = -f) and ||dx||_1, each the 1-norm
 * of the leading doubles of the md entries.  1 <= max_steps <= MDN_MAX_STEPS. */
mdn_status mdn_newton(mdn_ctx* ctx, int max_steps, double tol, int* steps_done, double* res_hist);

/* Copy the current series to x_out (device [K][C][n][d+1]). */
mdn_status mdn_get_series(const mdn_ctx* ctx, double* x_out);

/* Evaluate f at the current series into f_out (device [K][C][n][d+1]). */
mdn_status mdn_get_residual(mdn_ctx* ctx, double* f_out);

/* Evaluation and differentiation only (Section 5.1): f(x) into f_out and, when
 * A_out is not NULL, the Jacobian series into A_out (device
 * [K][C][d+1][n][n]).  x is a device series [K][C][n][d+1]. */
mdn_status mdn_evaluate(mdn_ctx* ctx, const double* x, double* f_out, double* A_out);

/* Linear solve only (Section 2, Eq. (eqToeplitz), with the Householder QR of
 * A0 of Section 5.3): dx with sum_{j<=k} A_j dx_{k-j} = b_k for k = 0..d.
 * A device [K][C][d+1][n][n], b and dx device [K][C][n][d+1].  Synchronises;
 * MDN_ESINGULAR for a zero pivot. */
mdn_status mdn_solve(mdn_ctx* ctx, const double* A, const double* b, double* dx);

/* Stated-accuracy variant of the forward substitution (the multiple double
 * arithmetic of Section 1 with the mixed-precision remark there, applied to
 * the right hand side updates of Section 5.4): stages k >= first_stage form
 * their block updates sum_{j>=1} A_j dx_{k-j} in `limbs` limbs, reading the
 * leading `limbs` doubles of every K-limb operand; the stage's right hand side
 * b_k, the solve dx_k = A0^{-1} r_k, the QR of A0, the residuals and the
 * evaluation stay in K limbs.  limbs must be K (variant off) or K/2 (K >= 2);
 * 1 <= first_stage, and first_stage > d switches the variant off.  Applies to
 * later mdn_newton and mdn_solve calls on the context.  Default: off. */
mdn_status mdn_set_late_updates(mdn_ctx* ctx, int first_stage, int limbs);

/* Staggered orders with the QR of A_0 once (Section 4: raise the order of
 * the series as the leading coefficients become correct; Section 5.3: factor
 * A_0 only in the first stage).  With first_steps >= 1, step s of later
 * mdn_newton calls works on the first L_s coefficients only: L_s = 1 for
 * s < first_steps (Newton on x_0 alone, with a QR of A_0 at every step), then
 * L := min(d+1, L + 1 + L/2) per step, every later step reusing the last
 * factorization.  The evaluation, the forward substitution and the update
 * skip the inactive coefficients; the norms of res_hist are over the active
 * ones, and a tolerance stops only at full order.  first_steps = 0 (default)
 * restores the plain method. */
mdn_status mdn_set_stagger(mdn_ctx* ctx, int first_steps);

/* Sampled residual monitor (Section 5.4 suggests the residuals of one or a
 * few random equations instead of all of them): later mdn_newton calls form
 * the monitor ||b - A dx||_1 on the `count` distinct rows listed (host
 * array, 0 <= rows[q] < n) and scale it by n / count, saving the A_0 dx_k
 * products of the other rows.  count = 0 (or n) restores all rows.  The
 * caller picks the rows (e.g. at random). */
mdn_status mdn_set_residual_rows(mdn_ctx* ctx, const int32_t* rows, int count);

/* Residual of the block lower triangular Toeplitz system of Eq.
 * (eqToeplitz) (the residual kernels of Sections 5.4 and 6):
 *   r_k = b_k - sum_{j=0..k} A_j dx_{k-j},   k = 0..d,
 * every entry rounded once to K limbs.  A device [K][C][d+1][n][n], b and dx
 * device [K][C][n][d+1]; r_out (device [K][C][n][d+1]) may be NULL.
 * *norm_out (host, may be NULL) receives the 1-norm of the leading doubles
 * of r (|re| or hypot), over the rows set by mdn_set_residual_rows (scaled by
 * n / count) or all rows.  Enqueued on the context's stream; synchronises to
 * read the norm.  Overwrites the context's per-entry residual magnitudes
 * (not the series). */
mdn_status mdn_residual(mdn_ctx* ctx, const double* A, const double* b, const double* dx, double* r_out,
                        double* norm_out);

/* out = s * a entry by entry (md multiplication; complex for C = 2): s is
 * one md value (device [K][C]), a and out device [K][C][count] (out may be
 * a).  Enqueued on the context's stream.  Used to scale a gradient by an
 * upstream md factor (the chain rule through an md-valued loss). */
mdn_status mdn_md_scale(mdn_ctx* ctx, const double* s, const double* a, int64_t count, double* out);

/* Bound of every device wait of the context's dataflow kernels (the QR of A0
 * and the forward substitution wait on flags and counters that other warps
 * publish), in nanoseconds of wall time; default 2e9.  A wait that runs out
 * records MDN_ETIMEOUT in the status word and its kernel returns, so the
 * synchronising call reports MDN_ETIMEOUT and the context stays usable.
 * limit_ns >= 1. */
mdn_status mdn_set_wait_limit_ns(mdn_ctx* ctx, int64_t limit_ns);

/* Adjoint of the converged series (real systems).  At a solution,
 * f(x(c), c) = 0 mod t^{d+1}, so the gradient of a loss L(x) with respect to
 * the coefficient series is dL/dc = -lambda^T df/dc with J^T lambda = dL/dx,
 * J the block lower triangular Jacobian of Eq. (eqToeplitz) at x.  J^T is
 * block upper triangular: lambda_k = A_0^{-T} (g_k - sum_{j>=1} A_j^T
 * lambda_{k+j}) for k = d..0, with A_0^{-T} from the Householder QR of A_0
 * (Section 5.3); then grad c_{m,j} = -sum_{k>=j} lambda_{eq(m),k}
 * [t^{k-j}] prod_{v in m} x_v (the products are recomputed).
 *   x: device [K][1][n][d+1], the series (normally mdn_newton's result);
 *   g: device [K][1][n][d+1], dL/dx as md values;
 *   grad_out: device [K][1][M][d+1].
 * MDN_EINVAL for complex data; MDN_ESINGULAR for a zero pivot of A_0.
 * Synchronises.  Overwrites the context's Jacobian and W (not x). */
mdn_status mdn_adjoint(mdn_ctx* ctx, const double* x, const double* g, double* grad_out);

/* The Fabry-ratio loss of a real series (Section 1.3: c_d / c_{d+1} of a
 * series tends to its nearest singularity),
 *   L = sum_i x_{i,d}^2 + x_{0,d-1} / x_{0,d},
 * into loss_out (device [K] limbs) and g_out = dL/dx (device
 * [K][1][n][d+1]).  Needs degree >= 1.  Enqueued on the context's stream. */
mdn_status mdn_fabry_loss(mdn_ctx* ctx, const double* x, double* loss_out, double* g_out);

/* Phases of a Newton step for mdn_profile(), after the kernel types of the
 * paper's Table 3 (Section 6.2): evaluation and differentiation
 * ("convolutions"), assembly of f and A, Householder QR with Q^H and back
 * substitution forming A0^{-1} ("qr", "qhb", "bs"), forward substitution
 * with the right hand side updates and residuals ("updates", "residuals"),
 * and the update of x with the norms of the step. */
#define MDN_NUM_PHASES 5
#define MDN_PHASE_EVALUATE 0
#define MDN_PHASE_ASSEMBLE 1
#define MDN_PHASE_QR 2
#define MDN_PHASE_FORWARD 3
#define MDN_PHASE_UPDATE 4

/* Device timers per phase.  enable = 1 clears the accumulators and starts
 * recording a CUDA event pair around every phase of later calls (on the
 * context's stream); enable = 0 stops recording, synchronises and writes the
 * accumulated milliseconds (ms_out) and kernel launch counts (launches_out)
 * per phase into host arrays of MDN_NUM_PHASES entries (either may be NULL). */
mdn_status mdn_profile(mdn_ctx* ctx, int enable, double* ms_out, int64_t* launches_out);

/* ---------------------------------------------------------------------------
 * Batched systems: many independent systems (each its own n, degree and
 * monomials, one K and C for all) solved in one persistent launch, each run
 * to its stop rule.  The paper's method (Section 2, with the kernels of
 * Sections 5.1-5.4) applied to every system; the batching itself, the work
 * queue and the stop rule are this library's.
 *
 * Packed layout.  System s has n_s equations and unknowns, D_s = degree_s+1
 * coefficients and M_s monomials; its monomials are the global indices
 * mono_s .. mono_s + M_s - 1 with mono_s = sum_{t<s} M_t.  Host arrays:
 * eq_of_monomial [Mtot] (equation within the system), var_ptr [Mtot+1] (CSR
 * offsets into var_idx, var_ptr[0] = 0), var_idx (variable within the
 * system; a repeat is a power).  Device arrays: coeff is the concatenation
 * over s of [K][C][M_s][D_s] blocks; const_term, x and f are concatenations
 * of [K][C][n_s][D_s] blocks, block s starting at sum_{t<s} K*C*n_t*D_t.
 *
 * Stop rule of mdn_batch_solve: ||f(x)||_inf <= tol before an update, or
 * ||dx||_inf <= tol * max(1, ||x||_inf) after one (leading doubles), or
 * max_steps updates.  steps_out[s] counts the updates applied; flags_out[s]
 * has bit 0 set when the stop rule was met, bit 1 for a zero pivot in the QR
 * of A_0 (system left at its last x), bit 2 for a non-finite value.
 *
 * Tiles: threads_per_block (multiple of 32, 128..1024, at least the largest
 * n) and blocks_per_sm (at most what the kernel's registers allow); 0 picks
 * 256 threads and the largest resident count.  Sizes: 1 <= n_s <= 128,
 * 0 <= degree_s <= 63, every monomial of at most 16 variables. */
typedef struct mdn_batch mdn_batch;

mdn_status mdn_batch_create(mdn_batch** out, int limbs, int is_complex, int count, const int32_t* n,
                            const int32_t* degree, const int32_t* n_monomials, int threads_per_block,
                            int blocks_per_sm);
/* Workspace for the system structure var_ptr (host [Mtot+1]); 0 on error. */
size_t mdn_batch_workspace_bytes(const mdn_batch* b, const int32_t* var_ptr);
/* Builds the tables on the host and copies them into the workspace (a device
 * buffer of ws_bytes >= mdn_batch_workspace_bytes, 256-byte aligned, borrowed
 * until mdn_batch_destroy).  coeff and const_term are borrowed device arrays.
 * Work is enqueued on `cuda_stream`. */
mdn_status mdn_batch_load(mdn_batch* b, const int32_t* eq_of_monomial, const int32_t* var_ptr,
                          const int32_t* var_idx, const double* coeff, const double* const_term, void* workspace,
                          size_t ws_bytes, void* cuda_stream);
/* f(x) of every system (device, packed); synchronises. */
mdn_status mdn_batch_evaluate(mdn_batch* b, const double* x, double* f_out);
/* Newton on every system from x0 (device, packed) into x (device, packed,
 * may equal x0), one persistent launch replayed from a CUDA graph; the host
 * arrays steps_out and flags_out [count] are filled; synchronises. */
mdn_status mdn_batch_solve(mdn_batch* b, const double* x0, double* x, int max_steps, double tol, int32_t* steps_out,
                           int32_t* flags_out);
/* The tiles in use. */
mdn_status mdn_batch_tiles(const mdn_batch* b, int* threads_per_block, int* blocks_per_sm);
const char* mdn_batch_last_error(const mdn_batch* b);
void mdn_batch_destroy(mdn_batch* b);

/* Size of the static device scratch of mdn_evaluate_static(). */
#define MDN_STATIC_SCRATCH_BYTES (2u << 20)

/* f(x(t)) without a context, a workspace or any device allocation.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory (plug-ins inside an application whose own pool
 * reserves the device memory up front, so that a cudaMalloc of theirs would
 * fail or fragment it; real-time loops that must not allocate after start-up,
 * since cudaMalloc can block on the device).  The scratch of the evaluation lives in
 * one file-scope device array of MDN_STATIC_SCRATCH_BYTES that every GPU
 * loading the library keeps until the process exits.
 *   All pointers are device pointers in the layouts above: eq_of_monomial [M],
 *   var_ptr [M+1], var_idx [n_var_refs], coeff [K][C][M][d+1], const_term and
 *   x [K][C][n][d+1]; f_out receives [K][C][n][d+1].
 * The call looks up the array's device address on its first use on a device
 * (cudaGetSymbolAddress, with that device current), so that first call should
 * come before any stream capture.  It returns MDN_ETOOLARGE when
 * 8 * (32 + n * 2 * K * C * (d+1)) bytes exceed MDN_STATIC_SCRATCH_BYTES,
 * MDN_EINVAL for bad sizes or an index out of range (eq_of_monomial,
 * var_ptr and var_idx, checked on the device); every call ends by
 * synchronising the stream to read that check.  All calls share the array
 * and it keeps the last call's contents: calls whose kernels overlap on the
 * GPU race.  No cudaMalloc, cudaFree or allocating routine is called. */
mdn_status mdn_evaluate_static(int limbs, int is_complex, int n, int degree, int n_monomials, int n_var_refs,
                               const int32_t* eq_of_monomial, const int32_t* var_ptr, const int32_t* var_idx,
                               const double* coeff, const double* const_term, const double* x, double* f_out,
                               void* cuda_stream);

/* The product schedule that the evaluation runs for one monomial of k
 * variables (Section 5.1: the three columns of forward products
 * F_j = F_{j-1} x_j, backward products B_j = B_{j-1} x_{k-j+1} and cross
 * products F_{p} B_{k-1-p}; the coefficient series c enters as F_0, so a
 * monomial with k >= 2 costs 3k-3 products, the paper's 3k-5 plus two).
 * Host only: no CUDA call, no device memory; it exposes the table that
 * mdn_load_system uploads so that host tests can execute it symbolically.
 *   k: 1..4096 variables; groups: 1..32 products that one warp runs at once.
 *   *n_waves receives the number of waves.  With ops non-NULL, ops receives
 *   n_waves * groups records of four int32 (op, destination, a, b): op 0 is
 *   an idle group, 1 a truncated product dst = a * b, 2 a copy dst = a; a
 *   slot is kind << 16 | index with kind 1 the coefficient c, 2 the input
 *   x_{index+1} (position in the monomial), 3 F_index, 4 B_index, 5 the
 *   value and 6 the partial with respect to position index.  capacity is the
 *   number of records ops holds; fewer than needed returns MDN_EINVAL.
 * Products of one wave read only slots written by earlier waves. */
mdn_status mdn_ed_schedule(int k, int groups, int32_t* ops, int capacity, int* n_waves);

/* Synchronise the context's stream and return the device status as an
 * mdn_status (MDN_OK when no device condition was raised). */
mdn_status mdn_status_word(mdn_ctx* ctx);

/* Message of the last failure on ctx (never NULL; "" when none). */
const char* mdn_last_error(const mdn_ctx* ctx);

/* Release the context (host memory only; device buffers stay the caller's). */
void mdn_destroy(mdn_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MDNEWTON_H */
