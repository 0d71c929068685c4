// Internal declarations shared by the libipt translation units.
//
// Data layout in device memory (npad = n rounded up to 128, kpad = k rounded
// up to 256; every padded entry is zero so no kernel needs K-edge checks):
//   Drow  [npad x npad] row-major Delta (FP64 in IPT_PREC_F64, else FP32)
//   DT    [npad x npad] column-major FP32 Delta (FP32 and tensor-core modes:
//         the exact Delta E term of the epilogue, P = Delta E + Delta W)
//   Dh,Dl [npad x npad] row-major 16-bit (FP16 or BF16) split of r_j Delta_j.,
//         r_j a power-of-two row scale (rinv[j] = 1 / r_j)
//   Z0,Z1 [kpad x npad] column-major iterates (FP64 or FP32), ping-pong
//   Wh,Wl [kpad x npad] column-major 16-bit split of s_c W_.c, W = Z - E
//         (E = unit columns), s_c a power-of-two column scale (sinv[c] = 1/s_c);
//         rewritten by the pre-pass of every tensor-core evaluation
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/ipt.h"

namespace ipt {

constexpr int kRowPad = 128;  // npad multiple (tile M of every product kernel)
constexpr int kColPad = 256;  // kpad multiple (tile N of the tensor-core kernel)

// Validation flags (DevState::flags).
enum : int {
  FLAG_COL_RANGE = 1,
  FLAG_COL_DUP = 2,
  FLAG_THETA_NONFINITE = 4,
  FLAG_THETA_DEGENERATE = 8,
  FLAG_ZERO_PIVOT = 16,
  FLAG_CSR_INDEX = 32,  // CSR row bounds or a column index out of range
};

// Device-resident solver state: norm accumulators of the running evaluation,
// the controller's decisions and the history.  Written by the product
// kernels (accumulators, atomics) and by k_control (one thread).
struct DevState {
  double acc_inc2;  // sum (F - Z)^2
  double acc_z2;    // sum Z^2
  double acc_r2;    // sum R^2, R = M Z - Z Lambda
  double acc_pv2;   // sum (Delta V)^2 of this evaluation's product (tensor-core epilogue)
  double r0acc;     // sum of squared off-diagonal Delta entries of requested columns
  double inc, rho, prev_rho;
  double kappa;     // ||Delta V|| / ||V|| of the last product (staged schedule)
  double sv;        // bound on ||Z - Z_base|| of the current iterate (staged schedule)
  // Error model of the products (absolute, in the units of ||R||):
  double e_base;    // predicted error of the stored base product P_b (0 for Z_b = E)
  double pw_base;   // bound on ||Delta (Z_b - E)|| of the base iterate
  double e_rel;     // predicted |rho - rho_true| of the last tested evaluation
  double rho_best;  // smallest residual of a tested evaluation so far (0: none yet)
  int acc_based;    // the current base came from a compensated FP32 product
  int stall;        // consecutive tested evaluations without a 10 % better residual
  int pause;   // nonzero: the next evaluation needs a kernel the enqueued ones do not
               // run (1: compensated FP32; 2: the acceleration the staged Picard phase
               // hands over to); enqueued kernels return at entry until cleared
  int want_acc;  // accelerated staged solves: the next tested evaluation should re-base
                 // on a compensated FP32 product
  int measure;   // the next evaluation samples its product error (k_sample_exact)
  // Next operand written by the product's epilogue (staged Picard, device-chosen
  // operands): the epilogue of an evaluation that may be followed by another
  // writes the 16-bit split of V_next = F - Z_b(next) into the W set not being
  // read (wsel ^ 1), with one power-of-two scale for all columns chosen from
  // vb, and the partial sums of d of F over its 32-row groups.  The controller
  // then hands the set over (split_ready), and the next pre-pass only adds the
  // partials and sets the scale.
  double vb;         // bound on max |V_next| for the scale of the next epilogue's split
  int wsel;          // W set (0/1) the tensor-core product reads
  int split_ready;   // the set wsel, the d partials and wscale hold the current operand
  int fused;         // this evaluation's epilogue wrote the next operand
  int split_bad;     // ... but a scaled entry left the 16-bit range (or was not finite)
  float wscale;      // 1 / scale of the current operand (fused split)
  float wscale_next; // 1 / scale of the operand the epilogue is writing
  int epi_used;      // evaluations that ran on such an operand
  // The caller's output Z (device entry point): the controller predicts that
  // the next evaluation forms the returned iterate (write_out), its product
  // epilogue then also stores F into Z and records its evaluation index
  // (out_iter; -1 for none), so no copy is needed after the loop.
  int write_out;
  int out_iter;
  // The operand the next epilogue writes carries its lo part only when the
  // evaluation that reads it is predicted to run the split (3-pass) product
  // (write_lo); fused_lo records what that epilogue wrote.
  int write_lo;
  int fused_lo;
  double acc_dp2;  // sum of squared product errors at the sampled entries
  double acc_dpn;  // number of sampled entries
  double e_meas;   // the last sampled estimate of ||P - Delta Z||_F (safety included)
  int done;    // nonzero: stop; every later kernel of the solve returns at entry
  int status;  // ipt_status once done
  int stage;   // ipt_precision of the next evaluation
  int passes;  // product passes of the next evaluation: 0 (no product), 1 or 3
  int rebase;  // next evaluation stores P and becomes the new base
  int accurate;  // next evaluation's product error is small enough to stop on
  int iter;    // evaluations completed
  int cur;     // Z buffer (0..2) holding the current iterate
  int base;    // Z buffer of the base iterate Z_b, or -1 for Z_b = E (P_b = Delta E)
  int answer;  // Z buffer holding the returned iterate
  int flags;   // validation flags
  int timeout; // bounded device wait gave up (code of the waiting role)
  int stage_iters[2];
  // CSR active window (rows outside it are exactly zero in Z and in F):
  int band;            // largest |j - m| over the stored entries of M
  int z_lo, z_hi;      // every nonzero row of the current iterate lies in [z_lo, z_hi]
  int nz_lo, nz_hi;    // the same for the F this evaluation writes
  int win_lo, win_hi;  // rows [win_lo, win_hi) evaluated by the next product
  long long rows_eval; // rows the products evaluated so far
  double hist_inc[IPT_MAX_HISTORY];
  double hist_rho[IPT_MAX_HISTORY];
  int hist_stage[IPT_MAX_HISTORY];
};

// Arguments of the fused map epilogue shared by all product kernels.
template <typename T>
struct MapArgs {
  const T* Zin;          // current iterate, column-major [kpad x npad], leading dim ld
  T* Fout;               // F(Z), same layout
  const float* DT;       // column-major FP32 Delta (FP32 / tensor-core modes, else null)
  // Tensor-core epilogues: P = Pbase + Delta V with V = Z - Z_base.  Pbase is
  // DT indexed by cols[c] (Z_base = E) or a stored P indexed by c; Pout, when
  // set, receives P (the evaluation becomes the new base).
  const float* Pbase;
  int pbase_by_icol;
  float* Pout;
  const float* rinv;     // per-row inverse operand scale (tensor-core modes)
  const float* sinv;     // per-column inverse operand scale (tensor-core modes)
  const double* d;       // d_c = (Delta Z)_{cols[c], c}
  const int32_t* icol;   // cols[c]; -1 in padding columns
  const double* theta;   // FP64 theta (F64 path)
  const float* th_hi;    // FP32 hi/lo split of theta (FP32 paths)
  const float* th_lo;
  int64_t ld;            // npad
  int n, k;
  DevState* st;
  // Sampled product error: with psmp set (and, with dyn, the state's measure
  // flag), the epilogue stores P at the rows j = r * smp_stride + smp_off,
  // r < kSampleRows, into psmp[r * kpad + c]; k_sample_exact compares them with
  // compensated FP32 dot products.
  float* psmp;
  int smp_stride, smp_off, smp_kpad;
  // Device-chosen operands (tensor-core evaluations enqueued ahead of the
  // host): with dyn set, the kernels take the iterate zsel[cur], write F into
  // zsel[zbuf_free(cur, base)], read P_b from pstore (base >= 0) or DT by
  // cols[c] (Z_b = E), store P into pstore when rebase, and run the pass count
  // of the device state, all read from st at entry.
  T* zsel[3];
  float* pstore;
  int dyn;
  // Next operand (DevState::vb): with fuse set (and dyn), the epilogue writes the
  // split of F - Z_b(next) into wnh / wnl [wsel ^ 1] and, per column c and group
  // g of 32 rows, sum_{j in g} Delta_{cols[c], j} F_jc into dpart[c * dgroups + g]
  // (Drow row-major Delta; dgroups = npad / 32).
  int fuse;
  int fuse_bf16;  // the split's 16-bit type: BF16 (else FP16)
  uint16_t* wnh[2];
  uint16_t* wnl[2];
  double* dpart;
  int dgroups;
  const float* drow;
  // Host-buffer entry point: the tensor-core epilogue also stores F into the
  // caller's host output (column-major n x k, leading dimension host_ld; the
  // device address of mapped pinned memory) when this evaluation's F is
  // predicted to be the returned iterate, so its copy overlaps the product.
  T* host_f;
  int64_t host_ld;
  // Device entry point: the same store into the caller's Z (column-major n x k,
  // out_ld), made only by an evaluation whose state asks for it (dyn, write_out).
  T* out_z;
  int64_t out_ld;
};

// Device-chosen pre-pass operands (see MapArgs::dyn): with dyn set, Z is
// z[cur], Z_b is z[base] (none for base -1) and the lo split is written only
// for a 3-pass product, all read from the device state at entry.
struct DynZ {
  const float* z[3];
  int dyn;
  // fused next operand (DevState::split_ready): the W sets, and the partial
  // sums of d of the iterate written by the previous product's epilogue
  uint16_t* wh[2];
  uint16_t* wl[2];
  double* dpart;
  int dgroups;
};

// The Z buffer receiving F: neither the current iterate nor the base.
__host__ __device__ inline int zbuf_free(int cur, int base) {
  for (int b = 0; b < 3; ++b)
    if (b != cur && b != base) return b;
  return 0;
}

// Rows of each product whose entries are recomputed to estimate its error.
constexpr int kSampleRows = 16;

// ---------------------------------------------------------------- launchers
// setup (k_setup.cu)
void launch_theta(const void* M, int64_t ldm, int m_dtype, const double* theta_in, int n,
                  int npad, double* theta, float* th_hi, float* th_lo, DevState* st,
                  cudaStream_t s);
void launch_validate(const int32_t* cols, int n, int k, int kpad, const double* theta,
                     int32_t* icol, int* count, DevState* st, cudaStream_t s);
// The sparse path's form (one launch): cols[] checked and counted as above,
// the requested columns' row range [z_lo, z_hi] recorded, and the unit entries
// of Z0 = E written into the row-major n x kk iterate Z (zero elsewhere
// already); duplicates are flagged by the row pass (count[j] > 1).
void launch_validate_csr(const int32_t* cols, int n, int k, int kk, int32_t* icol, int* count,
                         void* Z, int zf64, DevState* st, cudaStream_t s);
void launch_form_delta(const void* M, int64_t ldm, int m_dtype, const double* theta, int n,
                       int npad, const int* count, void* Drow, int drow_f64, float* DT,
                       double* r0part, DevState* st, cudaStream_t s);
void launch_split_delta(const float* Drow, int npad, int bf16, uint16_t* Dh, uint16_t* Dl,
                        float* rinv, cudaStream_t s);
void launch_init_z(const void* z0, int64_t ldz0, int z0_dtype, const int32_t* icol, int n,
                   int k, int npad, int kpad, void* Z, int z_f64, DevState* st, cudaStream_t s);
void launch_lambda(const double* theta, const int32_t* icol, const double* d, int k,
                   double* lambda, cudaStream_t s);
void launch_copy_z(const void* Z, int z_f64, int64_t ld, int n, int k, void* out,
                   int64_t ldo, int out_f64, cudaStream_t s);
void launch_convert_m64(const void* M, int64_t ldm, int m_dtype, int n, int npad, double* M64,
                        cudaStream_t s);

// iteration pieces (k_iter.cu)
void launch_prepass(const void* Drow, const void* Z, int f64, int64_t ld, const int32_t* icol,
                    int kpad, double* d, DevState* st, cudaStream_t s);
// Wl == nullptr: the lo part is not written (a 1-pass product follows)
void launch_prepass_tc(const float* Drow, const float* Z, const float* Zbase, int64_t ld,
                       const int32_t* icol, int kpad, int bf16, double* d, uint16_t* Wh,
                       uint16_t* Wl, float* sinv, DevState* st, cudaStream_t s,
                       const DynZ& dz = DynZ{});
// The evaluation at Z = E with no product (P = Delta E exactly): F = E - G o Delta_{., cols}.
void launch_map_first(const MapArgs<float>& a, int npad, int kpad, double* d, double* part,
                      cudaStream_t s);
void launch_gemm_simt_f64(const double* Drow, const MapArgs<double>& a, int npad, int kpad,
                          cudaStream_t s);
// compensated != 0: two-level (FP32 partials of 32 products, TwoSum pairs) sums
void launch_gemm_simt_f32(const float* Drow, const MapArgs<float>& a, int npad, int kpad,
                          int compensated, cudaStream_t s);
void launch_residual_f64(const double* M64, const double* Z64, int64_t ld, const double* lam,
                         int n, int k, int npad, int kpad, double* acc, cudaStream_t s);
struct ControlArgs {
  double tol, diverge_bound, stage_switch;  // stage_switch: safety fraction of the staged rule
  int max_iter, stop, mode, k;
  int low_stage, high_stage;  // STAGED: the 1-pass stage and the split stage it switches to
  // Error model: a product of V = Z - Z_b errs by about u * ||Delta V||, u per kind
  // (1-pass 16-bit, 3-pass split 16-bit, FP32 SIMT, compensated FP32 SIMT); the
  // FP32 (FP64) iterate arithmetic adds about e_arith * (||R0|| + ||Delta (Z - E)||).
  double u_low = 0.0, u_high = 0.0, u_f32 = 0.0, u_acc = 0.0, e_arith = 0.0;
  int guard = 0;        // residual stop: only rho + predicted error <= tol stops the solve
  int escalate = 0;     // STAGED: re-base on a compensated FP32 product when the split
                        // product's base error is what keeps the residual from tol
  int pause_on_acc = 0; // STAGED, device-chosen operands: pause before such an evaluation
  int out_pred = 0;     // STAGED, device-chosen operands: predict the evaluation that
                        // forms the returned iterate (DevState::write_out)
  int accel_staged = 0; // accelerated staged solves: request that re-base (want_acc)
  int host_base = -2;   // host-driven evaluations: the base this one used (-1: E), or -2
                        // for the controller's own (staged Picard) base
  int host_rebase = 0;  // with host_base >= -1: this evaluation stored its P as the base
  int host_stage = -1;  // with host_base >= -1: the stage and pass count this one ran
  int host_passes = -1;
  int host_measure = -1;  // host-driven: 1 if this evaluation's product error was sampled
                          // (k_sample_exact), 0 if not; -1: as the device state says
  double measure_below = 0.0;  // non-staged solves: sample the next evaluation's product
                               // error once rho is predicted below this (0: never)
  double slow_ratio = 0.0;  // STAGED with an acceleration to hand over to: once a tested
                            // residual falls by less than this factor per evaluation,
                            // pause (pause = 2) so that the host continues with it
  int smp_rows = 0;  // sampled rows of the product error estimate (0: no sampling)
  int n_rows = 0;    // n
  int csr_n = 0;              // CSR solves: n (the window is clipped to [0, n)); 0 = dense
  int csr_window = 0;         // CSR: nonzero = evaluate only rows that can be nonzero
  int acx = 0;                // ACX: the iterate stays in buffer 0 (no ping-pong)
  double step_scale = 1.0;    // largest ||Z_{t+1} - Z_t|| / ||F(Z_t) - Z_t|| (damping: 2)
  int test = 1;               // 0: no stopping test at this evaluation (ACX inner ones)
  int next_cur = -1;          // with acx: the buffer of the next iterate (Anderson), -1 keep
};

// Learned-damping model (k_mlp.cu): 6 -> 64 -> 64 -> 1, FP16 parameters.
constexpr int kMlpInputs = 6, kMlpHidden = 64;
constexpr int kMlpParams = kMlpInputs * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden +
                           kMlpHidden + kMlpHidden + 1;
cudaError_t launch_mlp_forward(const void* params, const float* X, int B, float* alpha,
                               cudaStream_t s);
cudaError_t launch_mlp_grad(const void* params, const float* X, const float* target, int B,
                            float* grad, double* loss, cudaStream_t s);
cudaError_t launch_mlp_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float b1, float b2, float eps, int step, cudaStream_t s);
// Learned damping-and-mixing model (k_mlp.cu): 7 -> 64 -> 64 -> 2, outputs
// (alpha, gamma) per sample.
constexpr int kMixInputs = 7;
constexpr int kMixParams = kMixInputs * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden +
                           kMlpHidden + kMlpHidden * 2 + 2;
cudaError_t launch_mix_forward(const void* params, const float* X, int B, float* out,
                               cudaStream_t s);
cudaError_t launch_mix_grad(const void* params, const float* X, const float* target, int B,
                            float* grad, double* loss, cudaStream_t s);
cudaError_t launch_mix_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float b1, float b2, float eps, int step, cudaStream_t s);

// The FP32 map's division (k_diag.cu): q[i] = u[i] * recip_nr(gap[i]).
cudaError_t launch_conv_check(int64_t count, const double* x, float* hi, float* lo, float* f,
                              double* back, int32_t* ok, cudaStream_t s);
cudaError_t launch_recip_check(int64_t count, const float* gap, const float* u, float* q,
                               cudaStream_t s);
// Bounded-wait check (k_diag.cu): out[0] = 1 if the wait succeeded, out[1] = ns waited.
cudaError_t launch_wait_check(int arrive, uint64_t limit_ns, long long* out, cudaStream_t s);

// Anderson mixing in the solve (k_anderson.cu): per-solve state.
struct AndState {
  double best_rho;  // smallest residual seen
  int steps;        // evaluations processed
  int fallback;     // nonzero: Picard steps from now on
};
// After the evaluation g = F(z) (z_prev, g_prev: the previous pair): the
// per-column mixing weights and out = g - gamma (g - g_prev); `first` (no
// previous pair) only records the residual.
cudaError_t launch_anderson_step(const void* z, const void* g, const void* zp, const void* gp,
                                 void* out, int f64, int n, int k, int64_t ld, double* acc,
                                 double* gamma, AndState* as, DevState* st, int first,
                                 cudaStream_t s);

// Learned damping in the solve (k_damp.cu): per-solve state of the model's use.
struct DampState {
  double best_rho;  // smallest residual seen
  int steps;        // column histories recorded so far
  int fallback;     // nonzero: plain Picard steps from now on
};
// After an evaluation at z (buffer) with F in f: per-column increments and
// eigenvalues into the history, features, the model's alphas, and
// f <- z + alpha (f - z) (the next iterate).  acc: 2k FP64 (zero on entry, left zero); hinc: 3k
// floats; hlam: 3k FP64; X: 6k floats; alpha: k floats.
cudaError_t launch_damp_step(const void* z, void* f, int f64, int n, int k, int64_t ld,
                             const double* theta, const int32_t* icol, const double* d,
                             const void* model, double* acc, float* hinc, double* hlam,
                             float* X, float* alpha, DampState* ds, DevState* st,
                             cudaStream_t s);

// Learned damping and mixing in the solve (k_mix.cu): after an evaluation g = F(z)
// (zp, gp: the previous pair, or null at the first step) per-column statistics,
// history and features, the mixing model's (alpha, gamma) into ag (2k floats),
// and out <- z + alpha f - gamma ((z - zp) + alpha (f - fp)) (out: zp's buffer).
// acc: 4k FP64 (zero on entry, left zero); hinc: 3k floats; hlam: 3k FP64;
// X: 7k floats.
cudaError_t launch_mix_step(const void* z, const void* g, const void* zp, const void* gp,
                            void* out, int f64, int n, int k, int64_t ld, const double* theta,
                            const int32_t* icol, const double* d, const void* model,
                            double* acc, float* hinc, double* hlam, float* X, float* ag,
                            DampState* ms, DevState* st, cudaStream_t s);

// Batched solve (k_batched.cu): largest problem order n; problem size classes
// (n <= 64, <= 256, larger) each with their own output tile (32 or 64, host
// array `tiles`).
constexpr int kBatchMaxN = 1024;
constexpr int kBatchClasses = 3;
inline int batch_class_host(int64_t n) { return n <= 64 ? 0 : (n <= 256 ? 1 : 2); }
cudaError_t launch_batched(const float* M, const double* theta, const int64_t* m_off,
                           const int64_t* v_off, const int* nsz, const int* order, int count,
                           int64_t max_n2, double tol, int max_iter, int stop,
                           double diverge_bound, double* lambda, float* Z, int* status,
                           int* iters, float* scratch, int* queue, const int* tiles, int ctas,
                           cudaStream_t s);
// resident CTAs per SM of the batched FP32 kernel
int batched_ctas_per_sm();
// Batched solve with tensor-core products (k_batched_tc.cu; passes 3 or 1):
// a prologue launch (one CTA per problem) and the main launch (one CTA per
// SM).  ws holds ctas x batched_tc_workspace(max_n) bytes; prep holds
// batched_tc_prep_bytes(...) bytes, where tiles_total sums
// batched_tc_tile_bytes(n) over the problems (t_off: its prefix sums) and
// total_n2 sums n^2.
int64_t batched_tc_tile_bytes(int64_t n);
int64_t batched_tc_workspace(int64_t max_n);
int64_t batched_tc_prep_bytes(int64_t tiles_total, int64_t total_n2, int count, int64_t max_n);
cudaError_t launch_batched_tc(const float* M, const double* theta, const int64_t* m_off,
                              const int64_t* v_off, const int64_t* t_off, const int* nsz,
                              const int* order, int count, int64_t max_n, int64_t tiles_total,
                              int64_t total_n2, double tol, int max_iter, int stop,
                              double diverge_bound, double* lambda, float* Z, int* status,
                              int* iters, void* ws, void* prep, int* queue, int ctas, int passes,
                              cudaStream_t s);

// Alg. 3 extrapolation of order p (2 or 3) in place: z (buffer of the
// extrapolated iterate) from f1 = f(z), f2, f3 (column-major, leading dim ld).
// acc: 2 * k FP64 scratch (zero on entry, left zero); sigma: k FP64.
void launch_acx_combine(void* z, const void* f1, const void* f2, const void* f3, int f64, int p,
                        int n, int k, int64_t ld, int global, double* acc, double* sigma,
                        DevState* st, cudaStream_t s);
// The same for the sparse path's row-major n x kk iterates over the state's
// window rows (blocks: persistent grid); with `window` the window is then
// widened by the band (the extrapolated iterate's rows need it).
void launch_acx_combine_rm(void* z, const void* f1, const void* f2, const void* f3, int f64,
                           int p, int n, int k, int kk, int window, int global, double* acc,
                           double* sigma, DevState* st, int blocks, cudaStream_t s);
// pdl: programmatic dependent launch (the sparse loop's chain of launches)
void launch_control(DevState* st, ControlArgs a, cudaStream_t s, bool pdl = false);

// Sampled error of the product just computed (k_sample.cu): the exact
// (compensated FP32) Delta Z at the sample rows of psmp against the stored P,
// sum of squared differences into st->acc_dp2.  Z: the evaluation's iterate, or
// with dz.dyn the state's current buffer (and nothing is done unless
// st->measure).  Drow: FP32 row-major Delta.
// scratch: sample_scratch_bytes() of device memory whose trailing counters
// (the last kMaxBlocks ints) are zero before the first launch; every launch
// leaves them zero.
int64_t sample_scratch_bytes();
void launch_sample_exact(const float* Drow, const float* Z, const int32_t* icol, int n, int k,
                         int kpad, int64_t ld, const float* psmp, int stride, int off,
                         void* scratch, DevState* st, const DynZ& dz, cudaStream_t s);

// tensor-core product (k_tc_gemm.cu).  passes = 1 (Dh Wh) or 3 (+ Dh Wl + Dl Wh);
// bf16 selects BF16 operands, else FP16.  Returns a cudaError_t of the launch
// or of tensor-map encoding.
// mode: IPT_PRODUCT_SINGLE or IPT_PRODUCT_PAIR (AUTO = PAIR); PAIR falls back
// to SINGLE when npad / 128 is odd.
cudaError_t launch_gemm_tc(const uint16_t* Dh, const uint16_t* Dl, const uint16_t* Wh,
                           const uint16_t* Wl, const MapArgs<float>& a, int npad, int kpad,
                           int passes, int bf16, int mode, cudaStream_t s);

// sparse path (k_csr.cu): Z row-major n x kk, kk = k rounded up to 64
void launch_csr_rows(const int32_t* rowptr, const int32_t* colind, const void* vals, int v_dtype,
                     const double* theta_in, int n, int64_t nnz, const int* count, double* theta,
                     float* th_hi, float* th_lo, double* delta, double* part, int window,
                     DevState* st, cudaStream_t s);
void launch_csr_prepass(const int32_t* rowptr, const int32_t* colind, const void* vals,
                        int v_dtype, const double* delta, const int32_t* icol, int kk,
                        const void* Z, int f64, double* d, DevState* st, cudaStream_t s);
// One sparse evaluation: d (in the SpMM for kk <= 512 columns, else a separate
// pre-pass launch) and the SpMM + map.  With `ev` (4 events): ev[0], ev[1]
// around the separate pre-pass, ev[2], ev[3] around the SpMM.  Returns the
// number of kernel launches.
int launch_csr_evaluate(const int32_t* rowptr, const int32_t* colind, const void* vals,
                        int v_dtype, const double* delta, const double* theta,
                        const float* th_hi, const float* th_lo, const int32_t* icol, double* d,
                        int n, int k, int kk, const void* Zin, void* Fout, int f64, int nblk,
                        DevState* st, cudaStream_t s, const cudaEvent_t* ev = nullptr);
// adds ||M Z - Z Lambda||_F^2 (FP64) of the row-major iterate to *acc
void launch_csr_residual64(const int32_t* rowptr, const int32_t* colind, const void* vals,
                           int v_dtype, int n, int k, int kk, const void* Z, int f64,
                           const double* lam, double* acc, cudaStream_t s);
// rows [j_lo, n) of the row-major iterate into the caller's column-major Z
void launch_csr_out(const void* Z, int f64, int j_lo, int n, int k, int kk, void* out,
                    int64_t ldo, int out_f64, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while the previous kernel of its stream is still running; it runs
// griddep_wait() (which returns once that kernel has completed and its memory
// is visible; at once for a plain launch) before it touches any memory the
// earlier kernels read or write.  griddep_launch() lets the next such launch
// be scheduled early.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_int(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_int(int v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sums carried as an unevaluated FP32 pair hi + lo ("double-float"): the
// pair addition is Knuth's TwoSum of the high parts with the low parts added
// to its error term, then renormalised (Dekker's fast two-sum), worth ~44
// significant bits.  Reductions of many FP32 partials use it instead of FP64,
// whose pipe runs at a small fraction of the FP32 rate on this GPU.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float av = __fsub_rn(s, bv);
  const float err = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(b.hi, bv));
  const float e = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ F2 warp_sum(F2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const F2 w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = f2_add(v, w);
  }
  return v;
}
__device__ __forceinline__ double f2_value(F2 v) { return (double)v.hi + (double)v.lo; }
// Sum over the block (blockDim.x a multiple of 32, at most 1024) as FP32
// pairs; the total is valid in thread 0.  `sh` (32 pairs) must not be in use.
__device__ __forceinline__ F2 block_sum(F2 v, F2* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  F2 t{0.f, 0.f};
  if (w == 0) t = warp_sum(lane < nw ? sh[lane] : F2{0.f, 0.f});
  return t;
}

// Exact FP32 <-> FP64 conversions and the two-float split of a double built
// from the IEEE bit patterns with integer instructions.  On this GPU the
// conversion instructions run on the narrow FP64 pipe, which per-row setup
// passes over millions of rows would otherwise saturate.  Each returns ok =
// false outside the range it handles (zero is handled; subnormal, infinite or
// NaN inputs and results are not), and the caller then uses the hardware
// conversion; within the range the results equal the hardware's.
//
// FP64 -> FP32, round to nearest even (normal FP32 results and zero).
__device__ __forceinline__ float f64_to_f32_rn_bits(double x, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if ((b << 1) == 0ull) {
    ok = true;
    return __uint_as_float(sign);
  }
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  const unsigned m23 = (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rem = (unsigned)(b & 0x1fffffffu);  // the 29 bits below FP32's last
  unsigned em = ((unsigned)(e + 127) << 23) | m23;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) em += 1u;  // carry ok
  ok = e >= -126 && e <= 127 && em < 0x7f800000u;
  return __uint_as_float(sign | em);
}

// FP32 -> FP64 (exact; normal inputs and zero).
__device__ __forceinline__ double f32_to_f64_bits(float v, bool& ok) {
  const unsigned u = __float_as_uint(v);
  const unsigned e8 = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  ok = true;
  if ((u << 1) == 0u) return __longlong_as_double((long long)sign);
  ok = e8 != 0u && e8 != 0xffu;
  const unsigned long long bits = sign | ((unsigned long long)(e8 - 127u + 1023u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// x = hi + lo to ~2^-48 relative: hi = RN_f32(x), lo = RN_f32(x - hi); x - hi is
// the 29 low bits (minus 2^29 when hi rounded up) at x's exponent, exact in an
// int, so lo is that int rounded to FP32 and scaled by a power of two.
__device__ __forceinline__ void split_f64_bits(double x, float& hi, float& lo, bool& ok) {
  hi = f64_to_f32_rn_bits(x, ok);
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if (!ok || (b << 1) == 0ull) {
    lo = 0.f;
    return;
  }
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  const unsigned m23 = (unsigned)((b >> 29) & 0x7fffffu);
  const int rem = (int)(b & 0x1fffffffu);
  const bool up = rem > 0x10000000 || (rem == 0x10000000 && (m23 & 1u));
  const int r = up ? rem - (1 << 29) : rem;
  if (e - 52 < -126) {  // the remainder's scale is not a normal FP32 power of two
    ok = false;
    return;
  }
  const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);
  // signed in the integer, so that a zero remainder is +0 as x - hi gives it
  lo = __int2float_rn((b >> 63) ? -r : r) * scale;  // exact: scaling by a power of two
}

// Power-of-two operand scale s with mx * s in [2^13, 2^14): keeps scaled
// values inside FP16's range (max 65504) with headroom; exponent clamped to
// +-60 so products of two scales stay finite.  1 for zero / non-finite mx.
__device__ __forceinline__ float pow2_scale(float mx) {
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int ex;
  frexpf(mx, &ex);
  const int e = max(-60, min(60, 14 - ex));
  return ldexpf(1.f, e);
}

// 16-bit hi/lo split of x: hi = rn(x), lo = rn(x - hi), as raw bits.
__device__ __forceinline__ void split16(float x, bool bf16, uint16_t& hi, uint16_t& lo) {
  if (bf16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  } else {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  }
}

// theta_j - theta_i from the two-float split (hi + lo = theta to ~2^-48
// relative): hi differences of nearby values are exact (Sterbenz), so the
// gap keeps ~24 significant bits even when |theta| >> |theta_j - theta_i|.
__device__ __forceinline__ float gap2f(float hj, float lj, float hi, float li) {
  return (hj - hi) + (lj - li);
}

// 1/g for the FP32 map: the hardware reciprocal estimate refined by one
// Newton-Raphson step, r <- r + r (1 - g r), which roughly doubles its
// correct bits (error ~1 ulp; the quotient u * r stays within ~1.5 ulp of
// u / g).  Four instructions instead of an IEEE division's ~15, in the
// elementwise epilogues that run once per matrix entry.
__device__ __forceinline__ float recip_nr(float g) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(g));
  return fmaf(r, fmaf(-g, r, 1.f), r);
}

// The map of Eq. (dyn) at one entry (j, c), j != cols[c]:
//   u = Z_jc d_c - P_jc,  F_jc = u / (theta_j - theta_{i_c}),
//   R_jc = (theta_j - theta_{i_c}) Z_jc - u   (= (M Z - Z Lambda)_jc).
// At j == cols[c]: F = 1, R = 0.  FP64 divides exactly; FP32 multiplies by
// the refined reciprocal.
template <typename T>
__device__ __forceinline__ void map_entry(T z, T p, T dc, T gap, bool diag, T& f, T& r) {
  if (diag) {
    f = T(1);
    r = T(0);
  } else {
    T u = z * dc - p;
    if constexpr (sizeof(T) == 8) f = u / gap;
    else f = u * recip_nr(gap);
    r = gap * z - u;
  }
}

// theta_j == theta_{cols[c]} off the unit entry: the gap of Eq. (single_line_dyn)
// does not exist (Section 3 requires distinct unperturbed eigenvalues).
__device__ __forceinline__ void flag_degenerate(DevState* st) {
  atomicOr(&st->flags, FLAG_THETA_DEGENERATE);
}

}  // namespace ipt
