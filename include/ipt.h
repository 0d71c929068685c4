/*
 * ipt.h - C ABI of libipt, a GB300 (sm_103a) implementation of Iterative
 * Perturbation Theory (IPT): Kenmoe, Kriemann, Smerlak, Zadorin, "A fast
 * iterative algorithm for near-diagonal eigenvalue problems" (2020).
 *
 * Problem (Section 3): for an n x n real matrix M and a partition
 * M = D + Delta with D = diag(theta) (theta pairwise distinct), the
 * eigenvectors z_i normalised by z_i[i] = 1 are the fixed points of
 *     f_i(z) = e_i + g_i o (z (Delta z)_i - Delta z),        Eq. (single_line_dyn)
 * and all of them together the fixed points of
 *     F(Z)   = I + G o (Z D(Delta Z) - Delta Z),             Eq. (dyn)
 * with G_jk = 1/(theta_j - theta_k), G_jj = 0.  Alg. 1 / Alg. 2 iterate
 * Z <- F(Z) from Z = I and return Lambda = D(M Z).  This library applies the
 * map to k requested columns cols[0..k-1] (k = n: the full spectrum).
 *
 * Conventions shared by every entry point:
 *  - Pointers marked "device" are CUDA device memory owned by the caller;
 *    the library never frees them.  Pointers marked "host" are host memory.
 *  - Z (iterates, warm starts, results) is column-major n x k with leading
 *    dimension ldz >= n: entry (j, c) is Z[c*ldz + j], so column c (the
 *    eigenvector continued from e_{cols[c]}) is contiguous.
 *  - Dense M is row-major with leading dimension ldm >= n: M[j*ldm + m].
 *  - Calls are ordered on the handle's stream and synchronise it before
 *    returning; outputs are valid on return.  A handle serves one host
 *    thread at a time.
 *  - Errors are returned, never raised or aborted on.  Size, pointer and
 *    option errors are detected before any kernel runs; column and theta
 *    errors (checked on the device) before any output is written.  On
 *    IPT_MAXITER / IPT_DIVERGED the outputs hold the last iterate at which F
 *    was evaluated.
 */
#ifndef IPT_H
#define IPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  IPT_OK = 0,               /* stopping test met                                     */
  IPT_MAXITER = 1,          /* max_iter evaluations of F without meeting the test    */
  IPT_DIVERGED = 2,         /* non-finite increment/residual or ||Z||_F > bound*sqrt(k) */
  IPT_DEGENERATE_THETA = 3, /* theta non-finite, or theta_j == theta_{cols[c]}, j != cols[c]
                               (Section 3 requires simple unperturbed eigenvalues)   */
  IPT_INVALID_ARG = 4,      /* bad size, pointer, dtype, column index or option      */
  IPT_CUDA_ERROR = 5,       /* a CUDA runtime call failed                            */
  IPT_DEVICE_TIMEOUT = 6,   /* a bounded device-side wait gave up                    */
  IPT_UNSUPPORTED = 7,      /* valid request this build cannot serve                 */
  IPT_INACCURATE = 8        /* residual stop with a fixed product precision: the test held
                               in the product's arithmetic, but rho plus the predicted error
                               of that arithmetic exceeds tol (the outputs hold that iterate;
                               IPT_PREC_STAGED escalates instead)                     */
} ipt_status;

/* Element types of inputs and outputs. */
typedef enum { IPT_DTYPE_F64 = 0, IPT_DTYPE_F32 = 1 } ipt_dtype;

/* Arithmetic of the product Delta Z (the dominant step, Section 4.2).
 * Tensor-core forms split Z = E + W (E = unit columns) and add the Delta E
 * term exactly in FP32, so only Delta W is rounded; operands carry a
 * power-of-two scale per row of Delta and per column of W (exact, undone in
 * the epilogue) so FP16's 5-bit exponent never overflows. */
typedef enum {
  IPT_PREC_F64 = 0,    /* FP64 product and iterate (CUDA cores)                        */
  IPT_PREC_F32 = 1,    /* plain FP32: FP32 FMA product of Delta W, FP32 iterate         */
  IPT_PREC_BF16 = 2,   /* BF16 tensor-core product (tcgen05), FP32 accumulate/iterate  */
  IPT_PREC_BF16X3 = 3, /* split-BF16 x3 tensor-core product (hi*hi + hi*lo + lo*hi)    */
  IPT_PREC_STAGED = 4, /* Products of V = Z - Z_b against a base iterate Z_b whose
                          product P_b is known accurately (first E, P_b = Delta E):
                          1-pass FP16 while its predicted error is small against the
                          predicted next residual, else one split FP16 x3 product
                          whose P becomes the new base (BF16 / BF16 x3 with
                          ipt_options.staged_bf16).  Only evaluations whose predicted
                          product error is below tol / 10 may declare convergence   */
  IPT_PREC_FP16 = 5,   /* FP16 tensor-core product, FP32 accumulate/iterate            */
  IPT_PREC_FP16X3 = 6, /* split-FP16 x3 tensor-core product                            */
  IPT_PREC_F32C = 7    /* FP32 FMA product of Delta W with compensated sums: FP32
                          partials of 32 products added as FP32 pairs (TwoSum); the
                          staged schedule's accurate re-base                          */
} ipt_precision;

/* Stopping test. */
typedef enum {
  IPT_STOP_INCREMENT = 0, /* ||F(Z) - Z||_F / ||Z||_F <= tol (Alg. 1/2)                 */
  IPT_STOP_RESIDUAL = 1   /* rho(Z) = ||M Z - Z Lambda||_F / ||M Z0 - Z0 Lambda0||_F <= tol,
                             Z0 the unit columns e_{cols[c]}                           */
} ipt_stop;

typedef struct {
  int precision;        /* ipt_precision; default IPT_PREC_STAGED                          */
  int stop;             /* ipt_stop; default IPT_STOP_RESIDUAL                             */
  double diverge_bound; /* IPT_DIVERGED when ||Z||_F > diverge_bound*sqrt(k); default 1e8  */
  double stage_switch;  /* STAGED: a 1-pass product is used while its predicted error is
                           below stage_switch x the predicted next residual; default 0.1  */
  int staged_bf16;      /* STAGED: nonzero = BF16 / BF16 x3 stages instead of FP16 / FP16 x3 */
  int verify_fp64;      /* nonzero: recompute ||M Z - Z Lambda||_F of the result in FP64
                           (result.rho_fp64); adds one FP64 product                        */
  int record_timing;    /* nonzero: time the pre-pass and product kernels with CUDA events
                           on the handle's stream (result.*_ms)                            */
  const void* z0;       /* optional warm start (device, Z layout, dtype = z_dtype);
                           column c is rescaled so that z0[cols[c], c] = 1                 */
  int product_kernel;   /* dense tensor-core product kernel: IPT_PRODUCT_AUTO (default),
                           IPT_PRODUCT_SINGLE (one CTA per 128 x 256 tile) or
                           IPT_PRODUCT_PAIR (two CTAs per 256 x 256 tile, one paired MMA;
                           needs an even number of 128-row blocks, else SINGLE is used).
                           Results are identical; only speed differs                     */
  int accel;            /* IPT_ACCEL_NONE (default, the Picard update of Alg. 1/2),
                           IPT_ACCEL_DAMPED, IPT_ACCEL_ANDERSON (below; dense only) or
                           IPT_ACCEL_ACX (Alg. 3: each extrapolation evaluates
                           F at z, f(z) [, f^2(z)] and moves z by the order-3 / order-2
                           extrapolation, orders 3, 2, 3, 2, ...; the stopping test is made
                           at the extrapolated points; `iterations` counts evaluations).
                           With IPT_PREC_STAGED the products are FP16 x3 (BF16 x3 with
                           staged_bf16)                                                    */
  int acx_sigma;        /* ACX step length: 0 (default) one per column, 1 one for all     */
  const void* damping_model; /* IPT_ACCEL_DAMPED: the damping model's parameters (device,
                                FP16, IPT_DAMPING_PARAMS values, layout of
                                ipt_damping_forward); IPT_ACCEL_MIXING: the mixing
                                model's (IPT_MIXING_PARAMS, ipt_mixing_forward)           */
  int csr_window;       /* ipt_solve_csr: nonzero (default) = each product evaluates only the
                           rows that can be nonzero: the rows of the current iterate's
                           nonzero rows widened by the band max|j - m| of the stored
                           entries (exact: other rows of Z and F are zero).  0 = all rows */
  int epilogue_operand; /* STAGED tensor-core solves: nonzero (default) = each product's
                           epilogue, which holds F, also writes the next evaluation's
                           operand (the 16-bit split of F - Z_b at one power-of-two scale
                           for all columns, chosen from a bound on ||F - Z_b||_F with a
                           factor of 4 to the 16-bit range; an entry outside it falls
                           back to the pre-pass) and accumulates d_c of F, so the next
                           pre-pass only hands them over.  0 = the pre-pass re-reads F
                           and writes the operand with a scale per column.  Results
                           agree to rounding                                              */
} ipt_options;

/* Values of ipt_options.accel.  IPT_ACCEL_DAMPED: learned damping (no counterpart in
 * the paper, whose Section 5 points to fixed-point acceleration in general): after each
 * evaluation Z <- Z + alpha_c (F(Z) - Z), alpha_c in (0, 2) predicted per column by the
 * damping model from the column's increment-norm and Rayleigh-quotient-change history
 * (see ipt_damping_forward); plain Picard steps for the first three evaluations and
 * after a fallback (a residual above ten times the smallest seen).  Runs inside the
 * staged precision schedule.
 * IPT_ACCEL_ANDERSON: depth-one Anderson mixing per column (also outside the paper):
 * with g = F and f = g(z) - z, the next iterate is g(z_t) - gamma_c (g(z_t) - g(z_{t-1})),
 * gamma_c = <f_t - f_{t-1}, f_t> / ||f_t - f_{t-1}||^2 (0 where that vanishes); the first
 * step and every step after the same fallback are Picard steps.  Precision as for ACX. */
enum {
  IPT_ACCEL_NONE = 0,
  IPT_ACCEL_ACX = 1,
  IPT_ACCEL_DAMPED = 2,
  IPT_ACCEL_ANDERSON = 3,
  IPT_ACCEL_MIXING = 4  /* learned damping and mixing (also outside the paper): after
                           each evaluation z <- z + alpha f - gamma ((z - z_prev) +
                           alpha (f - f_prev)), f = F(z) - z, with (alpha_c, gamma_c)
                           per column from the mixing model (ipt_mixing_forward; its
                           parameters in ipt_options.damping_model) fed the damping
                           model's six history features and the least-squares
                           Anderson weight; Picard steps first and after the same
                           fallback as IPT_ACCEL_DAMPED.  gamma = 0 is the damped step,
                           alpha = 1 Anderson mixing.  Precision as for ACX.        */
};

/* Values of ipt_options.product_kernel. */
enum { IPT_PRODUCT_AUTO = 0, IPT_PRODUCT_SINGLE = 1, IPT_PRODUCT_PAIR = 2 };

#define IPT_MAX_HISTORY 128

typedef struct {
  int status;           /* ipt_status                                                     */
  int iterations;       /* evaluations of F (products with Delta)                         */
  int stage_iters[2];   /* evaluations with a 1-pass FP16/BF16 product, and with any other
                           product; the product-free first evaluation at Z = E (P = Delta E
                           exactly) counts in neither                                     */
  double increment;     /* ||F(Z) - Z||_F / ||Z||_F at the returned Z                     */
  double rho;           /* relative residual of the returned pair, in the product's
                           arithmetic                                                     */
  double rho_fp64;      /* same, recomputed in FP64 (verify_fp64), else -1                */
  double r0;            /* ||M Z0 - Z0 Lambda0||_F, the residual normaliser               */
  int kernel_launches;  /* CUDA kernels this call launched                                */
  int product_launches[2]; /* product kernel launches: [0] 1-pass (FP16/BF16/FP32/FP64),
                              [1] 3-pass (FP16 x3 / BF16 x3)                             */
  double product_ms[2]; /* their summed device time (record_timing), else 0               */
  double prepass_ms;    /* summed device time of the D(Delta Z) / operand-split pre-pass  */
  double setup_ms;      /* device time of the partition / validation / Z0 kernels (timing) */
  double finalize_ms;   /* device time of the Lambda / Z output kernels (timing)           */
  double wall_ms;       /* host wall-clock time of the whole call                         */
  int history_len;      /* min(iterations, IPT_MAX_HISTORY)                               */
  double hist_increment[IPT_MAX_HISTORY];
  double hist_rho[IPT_MAX_HISTORY];
  int hist_stage[IPT_MAX_HISTORY]; /* precision of each evaluation's product (ipt_precision),
                                      -1 for the product-free first evaluation           */
  long long rows_evaluated; /* ipt_solve_csr: rows the products evaluated, summed over
                               evaluations (n per evaluation without the active window)  */
  int acc_launches;     /* compensated FP32 product launches (IPT_PREC_F32C evaluations)  */
  double acc_ms;        /* their summed device time (record_timing), else 0               */
  double rho_error;     /* predicted |rho - rho_true| of the returned pair: the error model
                           of the products and of the iterate's arithmetic (residual
                           stop: IPT_OK means rho + rho_error <= tol)                    */
  int epilogue_operands; /* evaluations whose product operand and d were written by the
                            previous product's epilogue (ipt_options.epilogue_operand)  */
} ipt_result;

typedef struct ipt_handle ipt_handle;

/* Fill *opt with the defaults listed above. */
void ipt_options_default(ipt_options* opt);

/* Human-readable name of a status code (static string). */
const char* ipt_status_string(int status);

/* Create a handle bound to `stream` (a cudaStream_t; NULL = the legacy default
 * stream) on the current device.  The handle owns a grow-only device
 * workspace (sized by the largest problem seen) and nothing else. */
ipt_status ipt_create(ipt_handle** h, void* stream);

/* Release the handle and its workspace.  NULL is accepted. */
ipt_status ipt_destroy(ipt_handle* h);

/*
 * Dense solve, Alg. 2 (k = n) or Alg. 1 per column (k < n).
 *   n        matrix order, >= 1
 *   M        device, row-major n x n, element type m_dtype, leading dim ldm >= n
 *   theta    device, n doubles: the diagonal D of the partition; NULL = diag(M)
 *   k        number of requested columns, 1 <= k <= n
 *   cols     device, k distinct int32 in [0, n): requested e_i; NULL = 0..k-1
 *   tol      stopping tolerance (>= 0) for opt->stop
 *   max_iter maximum evaluations of F, >= 1
 *   opt      options; NULL = defaults
 *   lambda   device, k doubles out: Lambda_c = theta_{cols[c]} + (Delta Z)_{cols[c], c}
 *   Z        device out, n x k column-major (ldz >= n), element type z_dtype
 *   out      host, filled with status, counts, norms and history
 * Returns the status also stored in out->status.
 */
ipt_status ipt_solve_dense(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                           const double* theta, int64_t k, const int32_t* cols, double tol,
                           int max_iter, const ipt_options* opt, double* lambda, void* Z,
                           int64_t ldz, int z_dtype, ipt_result* out);

/*
 * ipt_solve_dense with HOST buffers: M, theta, cols, lambda and Z are host
 * pointers.  The call copies the inputs to the handle's workspace, solves, and
 * copies Lambda and Z back.  A pinned (page-locked, device-mapped) M is read in
 * place by the setup, which forms Delta from it over the host link (no staging
 * copy).  When Z's dtype is the iterate's (FP32, or FP64 with IPT_PREC_F64) and
 * no acceleration is asked for, the iterate predicted to be returned reaches Z
 * early: copied on a second stream while the evaluation that tests it runs, or,
 * for a pinned Z and a tensor-core product, stored into Z by the epilogue of the
 * product that forms it (predicted when the test two evaluations on is expected
 * to pass).  Z may then hold another iterate if the call ends with a status
 * other than IPT_OK, IPT_MAXITER or IPT_DIVERGED.  Every copy and store has
 * finished when the call returns; M and Z must not be changed meanwhile.
 */
ipt_status ipt_solve_dense_host(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                                const double* theta, int64_t k, const int32_t* cols, double tol,
                                int max_iter, const ipt_options* opt, double* lambda, void* Z,
                                int64_t ldz, int z_dtype, ipt_result* out);

/*
 * One evaluation of the map, Eq. (dyn): F = F(Z) for a given Z, with
 * lambda_c = theta_{cols[c]} + (Delta Z)_{cols[c], c}.  Arguments as in
 * ipt_solve_dense; Zin (device, read) and Fout (device, written) use the Z
 * layout with ldz and z_dtype; `precision` is an ipt_precision (STAGED is
 * invalid here).  norms (host, 3 doubles, may be NULL) receives
 * ||F - Z||_F, ||Z||_F and ||M Z - Z Lambda||_F in the product's arithmetic.
 */
ipt_status ipt_step_dense(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                          const double* theta, int64_t k, const int32_t* cols, int precision,
                          const void* Zin, void* Fout, int64_t ldz, int z_dtype, double* lambda,
                          double* norms);

/*
 * Sparse solve with M in CSR form (Section 6.1 workloads: a few extremal
 * eigenpairs of a large sparse near-diagonal matrix).
 *   rowptr device, n+1 int32; colind device, nnz int32 (0-based, any order
 *   within a row, no duplicates); vals device, nnz of v_dtype.  rowptr must
 *   start at 0, ascend and end at nnz, and colind lie in [0, n): a violation
 *   is found on the device before any product and returns IPT_INVALID_ARG.  The CSR
 *   holds all stored entries of M, diagonal ones included; Delta = M - diag(theta).
 *   theta  device, n doubles; NULL = diag(M) (0 where a row stores no diagonal)
 * Every other argument as in ipt_solve_dense.  Product arithmetic: FP32
 * (IPT_PREC_F32; IPT_PREC_STAGED, the option default, also selects it) or
 * FP64 (IPT_PREC_F64); other precisions return IPT_UNSUPPORTED.  A warm start
 * (opt->z0) is not accepted here (IPT_INVALID_ARG).  opt->accel may be
 * IPT_ACCEL_NONE or IPT_ACCEL_ACX (Alg. 3 as for dense M, on the row-major
 * iterates and the active window widened by the band after each extrapolation;
 * acx_sigma as there); the other accelerations return IPT_UNSUPPORTED.
 * verify_fp64 recomputes
 * ||M Z - Z Lambda||_F of the result in FP64 over all n rows from the stored
 * entries (result.rho_fp64).  n < 2^30, nnz < 2^31.
 */
ipt_status ipt_solve_csr(ipt_handle* h, int64_t n, int64_t nnz, const int32_t* rowptr,
                         const int32_t* colind, const void* vals, int v_dtype,
                         const double* theta, int64_t k, const int32_t* cols, double tol,
                         int max_iter, const ipt_options* opt, double* lambda, void* Z,
                         int64_t ldz, int z_dtype, ipt_result* out);

/*
 * Many independent dense problems, each solved by Alg. 2 (all n_p eigenpairs,
 * theta = the given partition or diag(M_p)) with its own stopping test, in
 * one persistent launch: the GPU takes the problems largest first and runs
 * every evaluation of a problem without host involvement.  The exact Delta E
 * term plus the product Delta W (W = Z - E): opt->precision IPT_PREC_BF16X3
 * runs it on the tensor cores as split-BF16 x3 (128 x 128 tiles), IPT_PREC_BF16
 * as one BF16 pass, anything else as an FP32 SIMT product; FP32 iterate.  The
 * tensor-core forms add a prologue launch before the persistent one (the
 * operands' BF16 tiles and the first evaluation, one block per problem) and
 * use Z as working memory while they run.
 *   count          number of problems (>= 1)
 *   n              HOST array of count problem orders, 1 <= n_p <= 1024
 *   M              device, FP32, the problems packed back to back: problem p is
 *                  row-major n_p x n_p at element offset sum_{q<p} n_q^2
 *   theta          device FP64, packed at offset sum_{q<p} n_q, or NULL = diag(M_p)
 *   tol, max_iter  as in ipt_solve_dense (max_iter per problem)
 *   opt            precision, stop and diverge_bound are used (NULL = defaults: FP32)
 *   lambda         device FP64, packed like theta (written)
 *   Z              device FP32, packed like M, each block column-major (column c =
 *                  eigenvector continued from e_c) (written)
 *   status, iters  device int32[count] (written): each problem's ipt_status and
 *                  evaluations of F
 *   out            host: status IPT_OK when every problem converged, else the
 *                  status of the first problem (by index) that did not;
 *                  iterations = the largest evaluation count; product_ms[0] =
 *                  the kernels' device time with record_timing
 * Returns out->status (argument errors before any launch: IPT_INVALID_ARG).
 */
ipt_status ipt_solve_batched(ipt_handle* h, int64_t count, const int64_t* n, const float* M,
                             const double* theta, double tol, int max_iter,
                             const ipt_options* opt, double* lambda, float* Z, int32_t* status,
                             int32_t* iters, ipt_result* out);

/*
 * Output tile (rows x columns of Delta Z held by a block) of ipt_solve_batched,
 * one per size class: n <= 64, n <= 256, n <= 1024.  Each class is tuned on
 * the handle the first time a batch holds problems of that class (both tiles,
 * 32 and 64, timed on up to 64 of its problems; the faster kept); a set value
 * skips the tuning.  The solve's copy of the schedule, queue reset and kernel
 * run as one CUDA graph, captured on the first call and replayed while the
 * orders, pointers, tolerances and tiles repeat.
 *   ipt_set_batched_tiles   tiles[3] host: 32, 64, or 0 = tune on first use
 *   ipt_get_batched_tiles   tiles[3] host (written): the tiles in use, 0 = not tuned yet
 * Both return IPT_INVALID_ARG for a NULL handle or array or another value.
 */
ipt_status ipt_set_batched_tiles(ipt_handle* h, const int32_t* tiles);
ipt_status ipt_get_batched_tiles(const ipt_handle* h, int32_t* tiles);

/*
 * Check of the failure path of the device-side waits.  Every wait of the
 * tensor-core product kernel on a shared-memory barrier gives up after a time
 * limit (2 s), records a timeout in the solve's device state and lets the
 * kernel drain and return, and the solve reports IPT_DEVICE_TIMEOUT.  This call
 * runs the same wait in a one-CTA kernel on the caller's stream (NULL = legacy
 * default stream) and synchronises that stream:
 *   arrive      nonzero: a second warp arrives on the barrier (the wait succeeds);
 *               0: nothing ever arrives (the wait must give up)
 *   limit_s     the wait's time limit in seconds, 0 < limit_s <= 10
 *   succeeded   host (written): 1 if the wait completed, 0 if it gave up
 *   waited_s    host (written, may be NULL): seconds the wait took
 * Returns IPT_INVALID_ARG for a bad limit or NULL `succeeded`, IPT_CUDA_ERROR on
 * a CUDA failure, else IPT_OK.  No GPU fault or hang is involved either way.
 */
ipt_status ipt_check_bounded_wait(int arrive, double limit_s, void* stream, int32_t* succeeded,
                                  double* waited_s);

/*
 * Check of the FP32 map's division (no counterpart in the paper, which fixes no
 * precision).  The FP32 epilogues form F = u / (theta_j - theta_{i_c}) as u times
 * the hardware reciprocal estimate of the gap refined by one Newton-Raphson step;
 * this call applies that same device function elementwise,
 *   quotient[i] = u[i] * refined_reciprocal(gap[i]),  i < count,
 * to device FP32 arrays, enqueued on `stream` (NULL = legacy default stream)
 * without synchronising, so that it can be compared with IEEE division.
 * Returns IPT_INVALID_ARG for count < 0 or a NULL array, IPT_CUDA_ERROR on a
 * launch error.
 */
ipt_status ipt_check_map_division(int64_t count, const float* gap, const float* u,
                                  float* quotient, void* stream);

/*
 * Check of the exact conversions the sparse setup pass builds from IEEE bit
 * patterns with integer instructions (no counterpart in the paper): for i < count,
 *   hi[i], lo[i]  the two-float split of x[i] (hi = x rounded to FP32, lo = x - hi
 *                 rounded to FP32),
 *   f[i]          x[i] rounded to FP32,
 *   back[i]       f[i] converted back to FP64,
 *   ok[i]         bit 0: the split, bit 1: the rounding, bit 2: the conversion back
 *                 were inside the range the integer forms handle (outside it the
 *                 solver uses the hardware conversion; the outputs are then
 *                 unspecified),
 * on device arrays, enqueued on `stream` without synchronising, so that they can
 * be compared with the hardware conversions.  Returns IPT_INVALID_ARG for
 * count < 0 or a NULL array, IPT_CUDA_ERROR on a launch error.
 */
ipt_status ipt_check_conversions(int64_t count, const double* x, float* hi, float* lo,
                                 float* f, double* back, int32_t* ok, void* stream);

/*
 * The damping model of IPT_ACCEL_DAMPED and its training (no counterpart in the
 * paper).  A 6 -> 64 -> 64 -> 1 perceptron: h1 = tanh(x W1 + b1),
 * h2 = tanh(h1 W2 + b2), y = h2 W3 + b3, alpha = 2 / (1 + exp(-y)).  Parameters:
 * IPT_DAMPING_PARAMS FP16 values on the device, packed row-major in the order
 * W1[6][64], b1[64], W2[64][64], b2[64], W3[64][1], b3[1]; FP32 arithmetic.
 * Inputs x: rows of 6 FP32 features (device, B x 6 row-major; their definition is
 * the solver's, listed with IPT_ACCEL_DAMPED's kernels).  All calls are ordered on
 * `stream` (a cudaStream_t; NULL = the legacy default stream) and do not synchronise.
 *   ipt_damping_forward: alpha[b] for b < B (device FP32).
 *   ipt_damping_grad: ADDS the gradient of mean_b (alpha_b - target_b)^2 over the B
 *     samples to grad (device FP32[IPT_DAMPING_PARAMS]) and the mean to *loss
 *     (device FP64); the caller zeroes them.
 *   ipt_damping_adam: one Adam step (Kingma & Ba) on FP32 master parameters
 *     (device, IPT_DAMPING_PARAMS) with moments m, v (device FP32, zero at step 1),
 *     step >= 1; writes the FP16 parameters and zeroes grad.
 * Returns IPT_INVALID_ARG for a null pointer or B < 0, IPT_CUDA_ERROR on a launch error.
 */
#define IPT_DAMPING_PARAMS 4673
ipt_status ipt_damping_forward(int64_t B, const void* params, const float* x, float* alpha,
                               void* stream);
ipt_status ipt_damping_grad(int64_t B, const void* params, const float* x, const float* target,
                            float* grad, double* loss, void* stream);
ipt_status ipt_damping_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float beta1, float beta2, float eps, int step,
                            void* stream);

/*
 * The mixing model of IPT_ACCEL_MIXING and its training (no counterpart in the
 * paper).  A 7 -> 64 -> 64 -> 2 perceptron: h1 = tanh(x W1 + b1),
 * h2 = tanh(h1 W2 + b2), y = h2 W3 + b3, alpha = 2 / (1 + exp(-y0)),
 * gamma = 2 tanh(y1).  Parameters: IPT_MIXING_PARAMS FP16 values on the device,
 * packed row-major as W1[7][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2];
 * FP32 arithmetic.  Inputs: rows of 7 FP32 features (device, B x 7); outputs
 * and targets: rows (alpha, gamma) (device FP32, B x 2).  Calls are ordered on
 * `stream` (NULL = legacy default stream) and do not synchronise.
 *   ipt_mixing_forward: out[b] = (alpha_b, gamma_b) for b < B.
 *   ipt_mixing_grad: ADDS the gradient of mean_b ((alpha_b - t_b0)^2 + (gamma_b - t_b1)^2)
 *     to grad (device FP32[IPT_MIXING_PARAMS]) and the mean to *loss (device FP64).
 *   ipt_mixing_adam: one Adam step as ipt_damping_adam, on IPT_MIXING_PARAMS values.
 * Returns IPT_INVALID_ARG for a null pointer or B < 0, IPT_CUDA_ERROR on a launch error.
 */
#define IPT_MIXING_PARAMS 4802
ipt_status ipt_mixing_forward(int64_t B, const void* params, const float* x, float* out,
                              void* stream);
ipt_status ipt_mixing_grad(int64_t B, const void* params, const float* x, const float* target,
                           float* grad, double* loss, void* stream);
ipt_status ipt_mixing_adam(float* master, void* params, float* grad, float* m, float* v,
                           float lr, float beta1, float beta2, float eps, int step,
                           void* stream);

/*
 * ||M Z - Z Lambda||_F in FP64, allocating no device memory.  The paper has
 * no counterpart: this is a library service for callers that cannot call
 * cudaMalloc -- processes whose device memory belongs to another allocator
 * (e.g. a framework's caching pool, or a fixed memory budget) that forbids
 * side allocations, and loops where an allocation's implicit device
 * synchronisation is not acceptable.  Its only scratch is a fixed file-scope
 * device array of 16384 FP64 partial sums (128 KiB on every device that loads
 * the library, held until the library is unloaded).
 *   n, M, ldm, m_dtype   dense M as for ipt_solve_dense (device, row-major)
 *   k, Z, ldz, z_dtype   n x k column-major eigenvector block (device)
 *   lambda               device, k doubles
 *   out                  device, 1 double: the norm is written there
 *   stream               cudaStream_t the two kernels are enqueued on (NULL =
 *                        legacy default stream); the call does not synchronise
 * Limit: ceil(n/64) * ceil(k/64) <= 16384 (e.g. n = k = 8192); larger sizes
 * return IPT_UNSUPPORTED without launching anything.  A CUDA error already
 * pending on the calling thread returns IPT_CUDA_ERROR without launching and
 * is left pending for the caller.  The first call on a device (and the first
 * after a cudaDeviceReset) looks up the array's device address; make that
 * first call before any stream capture begins.  All calls share the array:
 * calls whose kernels overlap on the GPU (different streams, no ordering)
 * race on it and may return wrong norms.  Nothing in the array needs to start
 * at zero; each call overwrites the slots it reads.
 */
ipt_status ipt_residual_dense_noalloc(int64_t n, const void* M, int64_t ldm, int m_dtype,
                                      int64_t k, const void* Z, int64_t ldz, int z_dtype,
                                      const double* lambda, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IPT_H */
