// C ABI of libipt (declared in include/ipt.h): argument validation, the
// handle's workspace, and the host loop that drives Alg. 2 on the device.
//
// Per evaluation of F the host enqueues  d = D(Delta Z)  ->  product + map
// epilogue  ->  k_control,  then reads the controller's few words back.
// Every kernel returns at entry once the controller has set `done`.
#include "ipt_internal.cuh"

#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

using namespace ipt;

namespace {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

cudaError_t ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.cap = bytes;
  return e;
}

// Sparse solves enqueue this many evaluations per host synchronisation.
constexpr int kCsrChunk = 4;
// Dense tensor-core solves (device-chosen operands) likewise.
constexpr int kDenseChunk = 6;
constexpr int kEvbSlots = kDenseChunk > kCsrChunk ? kDenseChunk : kCsrChunk;
// Accumulation term of the split products' error model (see set_error_model).
constexpr double kSplitAccum = 0.66;
// Staged accelerated solves hand over to the acceleration once a tested residual
// falls by less than this factor per evaluation.
constexpr double kHandoverRatio = 0.25;

}  // namespace

struct ipt_handle {
  cudaStream_t s = nullptr;
  int dev = 0;
  Buf drow, dt, dh, dl, z[5], pbuf, wh, wl, rinv, sinv;  // z[4]: accelerated solves' base
  Buf smp;                          // sampled product entries (error estimate)
  float* host_f = nullptr;          // host entry point: the next tensor-core epilogue also
  int64_t host_ld = 0;              // stores F here (device address of the host output)
  float* out_z = nullptr;           // device entry point: the caller's Z, stored by the
  int64_t out_ld = 0;               // epilogue the controller picks (DevState::write_out)
  Buf wh2, wl2, dpart;              // staged Picard: the second W set and the partial sums
                                    // of d, both written by the product's epilogue
  Buf acx_d, acx_acc, acx_sigma;    // ACX: d of the inner evaluations, step-length sums, steps
  Buf damp;                         // learned damping: history, features, alphas, state
  Buf mix;                          // learned mixing: statistics, history, features, outputs
  Buf bmeta, bscratch;              // batched: schedule and offsets, per-CTA iterate pairs
  int btiles[kBatchClasses] = {};   // batched: tuned output tile per size class (0 = untuned)
  cudaStream_t gs = nullptr;        // batched: capture stream (the handle's may be the legacy one)
  cudaGraph_t bgraph = nullptr;     // batched: captured schedule copy + queue reset + kernel
  cudaGraphExec_t bexec = nullptr;
  uint64_t bkey = 0;                // hash of everything the captured graph depends on
  void* hmeta = nullptr;            // pinned staging of the batched schedule
  size_t hmeta_cap = 0;
  int* hstat = nullptr;             // pinned copy of per-problem statuses and counts
  size_t hstat_cap = 0;
  Buf theta, thh, thl, icol, count, d, st, r0part;
  Buf m64, z64, racc;
  Buf delta, cpart;                 // sparse path: delta_j = M_jj - theta_j, r0 partials
  Buf hM, hTheta, hCols, hLam, hZ;  // device staging of the host-buffer entry point
  DevState* hst = nullptr;          // pinned mirror of the controller's words
  DevState* hinit = nullptr;        // pinned initial controller words of a solve
  cudaEvent_t ev[8] = {};           // pre-pass / product / setup / finalize brackets
  cudaEvent_t evb[4 * kEvbSlots] = {};  // per-evaluation brackets of an enqueued chunk
  cudaStream_t cs = nullptr;        // host-buffer entry point: device-to-host copy stream
  cudaEvent_t zready = nullptr;     // an iterate is complete on the solve stream
  cudaEvent_t zcopied[3] = {};      // the last copy out of Z buffer b has finished
  int launches = 0;                 // kernels launched by the current call
  bool e_pending = false;           // Z buffer 0 does not hold the unit columns yet
  // Sparse path: Z buffers 0 and 1 are zero outside rows [csr_dirty_lo, csr_dirty_hi)
  // for the row-major layout (csr_n, csr_kk, csr_es) at these addresses; csr_n < 0
  // = unknown contents.
  int csr_n = -1, csr_kk = 0, csr_es = 0, csr_dirty_lo = 0, csr_dirty_hi = 0;
  void* csr_z[2] = {nullptr, nullptr};
};

namespace {

constexpr size_t kStateHead = offsetof(DevState, hist_inc);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return IPT_CUDA_ERROR; \
  } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

inline bool tensor_core(int prec) {
  return prec == IPT_PREC_BF16 || prec == IPT_PREC_BF16X3 || prec == IPT_PREC_STAGED ||
         prec == IPT_PREC_FP16 || prec == IPT_PREC_FP16X3;
}
inline bool bf16_operands(int prec, bool staged_bf16) {
  return prec == IPT_PREC_BF16 || prec == IPT_PREC_BF16X3 ||
         (prec == IPT_PREC_STAGED && staged_bf16);
}

// Problem geometry and buffer plan for one dense solve / step.
struct Plan {
  int n, k, npad, kpad, prec;
  bool f64;     // FP64 iterate and product
  bool tc;      // tensor-core buffers
  bool bf16;    // tensor-core operands are BF16 (else FP16)
  bool dt;      // column-major FP32 Delta (W-form epilogues)
  bool staged;  // third Z buffer and stored-P buffer (base re-use)
  int product_kernel = IPT_PRODUCT_AUTO;  // tensor-core product kernel variant
  bool acx = false;  // four Z buffers (z, f, f^2, f^3) and the extrapolation scratch
  bool acx_base = false;  // accelerated staged solve: fifth Z buffer (the base) and P_b
  bool damped = false;  // learned damping buffers
  bool mixing = false;  // learned mixing buffers
  bool epi_operand = false;  // staged Picard: the product's epilogue writes the next operand
};

// the sampled P entries, then (256-byte aligned) the estimator's scratch
inline size_t smp_scratch_off(const Plan& p) {
  return ((size_t)kSampleRows * p.kpad * 4 + 255) / 256 * 256;
}

ipt_status check_dense_args(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                            int64_t k, int prec, int64_t ldz, int z_dtype) {
  if (!h || !M) return IPT_INVALID_ARG;
  if (n < 1 || n > (1 << 20) || k < 1 || k > n || ldm < n || ldz < n) return IPT_INVALID_ARG;
  if (m_dtype != IPT_DTYPE_F64 && m_dtype != IPT_DTYPE_F32) return IPT_INVALID_ARG;
  if (z_dtype != IPT_DTYPE_F64 && z_dtype != IPT_DTYPE_F32) return IPT_INVALID_ARG;
  if (prec < IPT_PREC_F64 || prec > IPT_PREC_F32C) return IPT_INVALID_ARG;
  return IPT_OK;
}

// Learned-mixing scratch: acc (4k FP64), lam history (3k FP64), increment
// history (3k FP32), features (7k FP32), model outputs (2k FP32), state.
inline size_t mix_bytes(int kpad) { return (size_t)kpad * (32 + 24 + 12 + 28 + 8) + 64; }

ipt_status alloc_dense(ipt_handle* h, const Plan& p) {
  const size_t nn = (size_t)p.npad * p.npad, kn = (size_t)p.kpad * p.npad;
  const size_t ez = p.f64 ? 8 : 4;
  CK(ensure(h->drow, nn * ez));
  CK(ensure(h->z[0], kn * ez));
  CK(ensure(h->z[1], kn * ez));
  if (p.staged) {
    CK(ensure(h->z[2], kn * ez));
    CK(ensure(h->pbuf, kn * 4));
  }
  if (p.damped) {
    CK(ensure(h->acx_acc, (size_t)p.kpad * 2 * 8));
    CK(ensure(h->damp, (size_t)p.kpad * (3 * 8 + 3 * 4 + 6 * 4 + 4) + 64));
  }
  if (p.mixing) CK(ensure(h->mix, mix_bytes(p.kpad)));
  if (p.acx_base) {
    CK(ensure(h->z[4], kn * ez));
    CK(ensure(h->pbuf, kn * 4));
  }
  if (p.acx) {
    CK(ensure(h->z[2], kn * ez));
    CK(ensure(h->z[3], kn * ez));
    CK(ensure(h->acx_d, (size_t)p.kpad * 2 * 8));
    CK(ensure(h->acx_acc, (size_t)p.kpad * 2 * 8));
    CK(ensure(h->acx_sigma, (size_t)p.kpad * 8));
  }
  if (p.dt) CK(ensure(h->dt, nn * 4));
  if (p.tc) {
    CK(ensure(h->dh, nn * 2));
    CK(ensure(h->dl, nn * 2));
    CK(ensure(h->wh, kn * 2));
    CK(ensure(h->wl, kn * 2));
    CK(ensure(h->rinv, (size_t)p.npad * 4));
    CK(ensure(h->sinv, (size_t)p.kpad * 4));
    CK(ensure(h->smp, smp_scratch_off(p) + (size_t)sample_scratch_bytes()));
    if (p.epi_operand) {
      CK(ensure(h->wh2, kn * 2));
      CK(ensure(h->wl2, kn * 2));
      CK(ensure(h->dpart, (size_t)p.kpad * (p.npad / 32) * 8));
    }
  }
  CK(ensure(h->theta, (size_t)p.npad * 8));
  CK(ensure(h->thh, (size_t)p.npad * 4));
  CK(ensure(h->thl, (size_t)p.npad * 4));
  CK(ensure(h->icol, (size_t)p.kpad * 4));
  CK(ensure(h->count, (size_t)p.npad * 4));
  CK(ensure(h->d, (size_t)p.kpad * 8));
  CK(ensure(h->st, sizeof(DevState)));
  // per-block partial sums: setup's ||R0||^2 and the first evaluation's norms
  CK(ensure(h->r0part, std::max((size_t)(p.npad / 32) * (p.npad / 32),
                                (size_t)p.kpad * ((p.npad / 4 + 255) / 256) * 3) * 8));
  return IPT_OK;
}

DevState* dst(ipt_handle* h) { return static_cast<DevState*>(h->st.p); }

// Sampled rows of the product-error estimate: j_r = r * stride + stride / 2.
inline int sample_stride(const Plan& p) { return p.npad / kSampleRows; }
inline int sample_rows(const Plan& p) {
  int r = 0;
  for (int q = 0; q < kSampleRows; ++q) r += q * sample_stride(p) + sample_stride(p) / 2 < p.n;
  return r;
}
void set_sampling(ipt_handle* h, const Plan& p, MapArgs<float>& a, bool on) {
  a.psmp = on ? (float*)h->smp.p : nullptr;
  a.smp_stride = sample_stride(p);
  a.smp_off = sample_stride(p) / 2;
  a.smp_kpad = p.kpad;
}


ipt_status status_from_flags(int flags) {
  if (flags & (FLAG_COL_RANGE | FLAG_COL_DUP | FLAG_ZERO_PIVOT | FLAG_CSR_INDEX))
    return IPT_INVALID_ARG;
  if (flags & (FLAG_THETA_NONFINITE | FLAG_THETA_DEGENERATE)) return IPT_DEGENERATE_THETA;
  return IPT_OK;
}

// Partition, validation and starting point; leaves the controller state
// initialised with the first stage.  z0 (optional) is copied into Z buffer 0,
// rescaled to z0[cols[c], c] = 1 when `rescale`.  With `sync_check` the
// validation flags are read back here; otherwise the caller reads them at
// its first synchronisation, before writing any output (every setup kernel
// is memory-safe on invalid columns or theta).
// Host destination of the returned iterate (host-buffer entry point): the
// iterate predicted to be returned is copied out to the host beside the
// evaluation that tests it.
struct HostOut {
  void* Z = nullptr;  // host, column-major n x k, ldz, the iterate's dtype
  int64_t ldz = 0;
  void* Zdev = nullptr;  // Z's device address (mapped pinned memory), else null
};

// Initial controller state: the first evaluation's stage, product passes
// (0 = product-free evaluation at Z = E), base and accuracy class.
struct FirstEval {
  int stage, passes, rebase, accurate;
  bool defer_e = true;  // the unit columns may be written only if returned
};

ipt_status setup_dense(ipt_handle* h, const Plan& p, const void* M, int64_t ldm, int m_dtype,
                       const double* theta, const int32_t* cols, const void* z0, int64_t ldz0,
                       int z0_dtype, bool rescale, FirstEval fe, bool sync_check) {
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  h->csr_n = -1;  // the dense path overwrites the shared Z buffers
  CK(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  {
    DevState& init = *h->hinit;  // pinned: the copy below is truly asynchronous
    memset(&init, 0, kStateHead);
    init.stage = fe.stage;
    init.passes = fe.passes;
    init.rebase = fe.rebase;
    init.accurate = fe.accurate;
    init.base = -1;
    init.out_iter = -1;
    CK(cudaMemcpyAsync(st, h->hinit, kStateHead, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemsetAsync(h->count.p, 0, (size_t)p.npad * 4, s));
  ipt_status v = IPT_OK;
  launch_theta(M, ldm, m_dtype, theta, p.n, p.npad, (double*)h->theta.p, (float*)h->thh.p,
               (float*)h->thl.p, st, s);
  launch_validate(cols, p.n, p.k, p.kpad, (const double*)h->theta.p, (int32_t*)h->icol.p,
                  (int*)h->count.p, st, s);
  h->launches += 3;
  CK(cudaGetLastError());
  if (sync_check) {
    CK(cudaMemcpyAsync(h->hst, st, kStateHead, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    v = status_from_flags(h->hst->flags);
    if (v != IPT_OK) return v;
  }
  launch_form_delta(M, ldm, m_dtype, (const double*)h->theta.p, p.n, p.npad,
                    (const int*)h->count.p, h->drow.p, p.f64 ? 1 : 0,
                    p.dt ? (float*)h->dt.p : nullptr, (double*)h->r0part.p, st, s);
  h->launches += 2;  // form_delta, sum of partials
  if (p.tc) {
    launch_split_delta((const float*)h->drow.p, p.npad, p.bf16 ? 1 : 0, (uint16_t*)h->dh.p,
                       (uint16_t*)h->dl.p, (float*)h->rinv.p, s);
    h->launches += 1;
  }
  if (p.tc) {
    // the error estimator's arrival counters start at zero (each launch leaves them so)
    CK(cudaMemsetAsync((char*)h->smp.p + smp_scratch_off(p), 0, (size_t)sample_scratch_bytes(),
                       s));
    // padding columns of the W operand stay zero (the pre-pass skips them)
    const size_t pad = (size_t)(p.kpad - p.k) * p.npad * 2;
    if (pad) {
      CK(cudaMemsetAsync((char*)h->wh.p + (size_t)p.k * p.npad * 2, 0, pad, s));
      CK(cudaMemsetAsync((char*)h->wl.p + (size_t)p.k * p.npad * 2, 0, pad, s));
    }
  }
  const size_t kn = (size_t)p.kpad * p.npad;
  const size_t ez = p.f64 ? 8 : 4;
  // Z buffers receive F only at rows < n of columns < k: zero the rest once
  // (buffer 0 too: with the deferred unit columns nothing else writes it before
  // an evaluation stores F there, and later pre-passes read every row of a column)
  for (int b = 0; b < (p.acx ? (p.acx_base ? 5 : 4) : p.staged ? 3 : 2); ++b) {
    if (p.npad > p.n)
      CK(cudaMemset2DAsync((char*)h->z[b].p + (size_t)p.n * ez, (size_t)p.npad * ez, 0,
                           (size_t)(p.npad - p.n) * ez, (size_t)p.kpad, s));
    if (p.kpad > p.k)
      CK(cudaMemsetAsync((char*)h->z[b].p + (size_t)p.k * p.npad * ez, 0,
                         (size_t)(p.kpad - p.k) * p.npad * ez, s));
  }
  h->e_pending = false;
  if (z0 && !rescale) {
    // exact copy (single evaluation at a caller-given Z)
    CK(cudaMemsetAsync(h->z[0].p, 0, kn * (p.f64 ? 8 : 4), s));
    launch_copy_z(z0, z0_dtype == IPT_DTYPE_F64, ldz0, p.n, p.k, h->z[0].p, p.npad, p.f64 ? 1 : 0,
                  s);
    h->launches += 1;
  } else if (!z0 && fe.passes == 0 && fe.defer_e) {
    // the product-free first evaluation knows Z = E without reading it: the
    // unit columns are written only if the solve returns that iterate
    h->e_pending = true;
  } else {
    launch_init_z(z0, ldz0, z0_dtype, (const int32_t*)h->icol.p, p.n, p.k, p.npad, p.kpad,
                  h->z[0].p, p.f64 ? 1 : 0, st, s);
    h->launches += 1;
  }
  CK(cudaGetLastError());
  if (sync_check) {
    CK(cudaMemcpyAsync(h->hst, st, kStateHead, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    v = status_from_flags(h->hst->flags);
    if (v != IPT_OK) return v;
  }
  return IPT_OK;
}

struct Timing {
  bool on = false;
  double product_ms[3] = {0.0, 0.0, 0.0};  // 1-pass, 3-pass, compensated FP32
  int product_launches[3] = {0, 0, 0};
  double prepass_ms = 0.0;
  double setup_ms = 0.0, finalize_ms = 0.0;
};

ipt_status ensure_events(ipt_handle* h) {
  for (int i = 0; i < 8; ++i)
    if (!h->ev[i]) CK(cudaEventCreate(&h->ev[i]));
  for (int i = 0; i < 4 * kEvbSlots; ++i)
    if (!h->evb[i]) CK(cudaEventCreate(&h->evb[i]));
  return IPT_OK;
}

// Buffer receiving F: neither the current iterate nor the base.
int free_buffer(int cur, int base) { return zbuf_free(cur, base); }

// One evaluation at Z buffer `cur`: d, product of V = Z - Z_base (in `passes`
// passes of arithmetic `stage`; 0 = product-free first evaluation at Z = E),
// map.  `rebase` stores P as the new base product.
// `out` >= 0 names the buffer receiving F (else the free one), `dv` the vector
// receiving d (else the handle's), `ev` the four timing events (else the handle's).
ipt_status evaluate(ipt_handle* h, const Plan& p, int cur, int base, int stage, int passes,
                    int rebase, Timing* tm, int out = -1, double* dv = nullptr,
                    cudaEvent_t* ev = nullptr, int measure = 0) {
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  const int nxt = out >= 0 ? out : free_buffer(cur, base);
  double* dd = dv ? dv : (double*)h->d.p;
  if (!ev) ev = h->ev;
  const bool t = tm && tm->on;
  bool ev3_done = false;
  if (t) CK(cudaEventRecord(ev[0], s));
  if (p.f64) {
    launch_prepass(h->drow.p, h->z[cur].p, 1, p.npad, (const int32_t*)h->icol.p, p.kpad,
                   dd, st, s);
    if (t) CK(cudaEventRecord(ev[1], s));
    MapArgs<double> a{};
    a.Zin = (const double*)h->z[cur].p;
    a.Fout = (double*)h->z[nxt].p;
    a.d = dd;
    a.icol = (const int32_t*)h->icol.p;
    a.theta = (const double*)h->theta.p;
    a.ld = p.npad;
    a.n = p.n;
    a.k = p.k;
    a.st = st;
    if (t) CK(cudaEventRecord(ev[2], s));
    launch_gemm_simt_f64((const double*)h->drow.p, a, p.npad, p.kpad, s);
  } else {
    MapArgs<float> a{};
    a.Zin = (const float*)h->z[cur].p;
    a.Fout = (float*)h->z[nxt].p;
    a.DT = (const float*)h->dt.p;
    a.d = dd;
    a.icol = (const int32_t*)h->icol.p;
    a.th_hi = (const float*)h->thh.p;
    a.th_lo = (const float*)h->thl.p;
    a.ld = p.npad;
    a.n = p.n;
    a.k = p.k;
    a.st = st;
    if (passes == 0) {
      // Z = E: P = Delta E exactly, no product (counted with the pre-pass time)
      launch_map_first(a, p.npad, p.kpad, dd, (double*)h->r0part.p, s);
      if (t) {
        CK(cudaEventRecord(ev[1], s));
        CK(cudaEventRecord(ev[2], s));
      }
    } else if (stage == IPT_PREC_F32 || stage == IPT_PREC_F32C) {
      // products of W = Z - E (base E, P_b = Delta E exact); the compensated one
      // may store its P as the new base
      launch_prepass(h->drow.p, h->z[cur].p, 0, p.npad, (const int32_t*)h->icol.p, p.kpad,
                     dd, st, s);
      if (t) CK(cudaEventRecord(ev[1], s));
      if (t) CK(cudaEventRecord(ev[2], s));
      a.Pout = rebase ? (float*)h->pbuf.p : nullptr;
      launch_gemm_simt_f32((const float*)h->drow.p, a, p.npad, p.kpad,
                           stage == IPT_PREC_F32C ? 1 : 0, s);
    } else {
      const float* zb = base >= 0 ? (const float*)h->z[base].p : nullptr;
      launch_prepass_tc((const float*)h->drow.p, (const float*)h->z[cur].p, zb, p.npad,
                        (const int32_t*)h->icol.p, p.kpad, p.bf16 ? 1 : 0, dd,
                        (uint16_t*)h->wh.p,
                        passes == 1 ? nullptr : (uint16_t*)h->wl.p,  // lo part for 3 passes
                        (float*)h->sinv.p, st, s);
      if (t) CK(cudaEventRecord(ev[1], s));
      a.rinv = (const float*)h->rinv.p;
      a.sinv = (const float*)h->sinv.p;
      a.Pbase = base >= 0 ? (const float*)h->pbuf.p : (const float*)h->dt.p;
      a.pbase_by_icol = base >= 0 ? 0 : 1;
      a.Pout = rebase ? (float*)h->pbuf.p : nullptr;
      set_sampling(h, p, a, measure != 0);
      a.host_f = h->host_f;
      a.host_ld = h->host_ld;
      if (t) CK(cudaEventRecord(ev[2], s));
      CK(launch_gemm_tc((const uint16_t*)h->dh.p, (const uint16_t*)h->dl.p,
                        (const uint16_t*)h->wh.p, (const uint16_t*)h->wl.p, a, p.npad, p.kpad,
                        passes, p.bf16 ? 1 : 0, p.product_kernel, s));
      if (t) CK(cudaEventRecord(ev[3], s));  // the product kernel alone
      ev3_done = true;
      if (measure) {
        launch_sample_exact((const float*)h->drow.p, (const float*)h->z[cur].p,
                            (const int32_t*)h->icol.p, p.n, p.k, p.kpad, p.npad,
                            (const float*)h->smp.p, sample_stride(p), sample_stride(p) / 2,
                            (char*)h->smp.p + smp_scratch_off(p), st, DynZ{}, s);
        h->launches += 1;
      }
    }
  }
  CK(cudaGetLastError());
  if (t && !ev3_done) CK(cudaEventRecord(ev[3], s));
  h->launches += 2;
  return IPT_OK;
}

// One tensor-core evaluation whose operands the device chooses (MapArgs::dyn,
// DynZ): the current iterate, the base, the pass count and the re-base come
// from the controller's state, so the host can enqueue evaluations without
// reading its choices.  Events ev[0..3] as in evaluate().
ipt_status evaluate_dyn(ipt_handle* h, const Plan& p, Timing* tm, cudaEvent_t* ev) {
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  const bool t = tm && tm->on;
  if (t) CK(cudaEventRecord(ev[0], s));
  DynZ dz{};
  for (int b = 0; b < 3; ++b) dz.z[b] = (const float*)h->z[b].p;
  dz.dyn = 1;
  // staged Picard: the product's epilogue writes the next operand into the other
  // W set (DevState::vb); the pre-pass then only hands over d and the scale
  const bool fuse = p.epi_operand && h->wh2.p && h->wl2.p && h->dpart.p;
  if (fuse) {
    dz.wh[0] = (uint16_t*)h->wh.p;
    dz.wl[0] = (uint16_t*)h->wl.p;
    dz.wh[1] = (uint16_t*)h->wh2.p;
    dz.wl[1] = (uint16_t*)h->wl2.p;
    dz.dpart = (double*)h->dpart.p;
    dz.dgroups = p.npad / 32;
  }
  launch_prepass_tc((const float*)h->drow.p, nullptr, nullptr, p.npad, (const int32_t*)h->icol.p,
                    p.kpad, p.bf16 ? 1 : 0, (double*)h->d.p, (uint16_t*)h->wh.p,
                    (uint16_t*)h->wl.p, (float*)h->sinv.p, st, s, dz);
  if (t) {
    CK(cudaEventRecord(ev[1], s));
    CK(cudaEventRecord(ev[2], s));
  }
  MapArgs<float> a{};
  a.DT = (const float*)h->dt.p;
  a.d = (const double*)h->d.p;
  a.icol = (const int32_t*)h->icol.p;
  a.th_hi = (const float*)h->thh.p;
  a.th_lo = (const float*)h->thl.p;
  a.rinv = (const float*)h->rinv.p;
  a.sinv = (const float*)h->sinv.p;
  a.ld = p.npad;
  a.n = p.n;
  a.k = p.k;
  a.st = st;
  for (int b = 0; b < 3; ++b) a.zsel[b] = (float*)h->z[b].p;
  a.pstore = p.staged ? (float*)h->pbuf.p : nullptr;
  a.dyn = 1;
  if (fuse) {
    a.fuse = 1;
    a.fuse_bf16 = p.bf16 ? 1 : 0;
    a.wnh[0] = (uint16_t*)h->wh.p;
    a.wnl[0] = (uint16_t*)h->wl.p;
    a.wnh[1] = (uint16_t*)h->wh2.p;
    a.wnl[1] = (uint16_t*)h->wl2.p;
    a.dpart = (double*)h->dpart.p;
    a.dgroups = p.npad / 32;
    a.drow = (const float*)h->drow.p;
  }
  set_sampling(h, p, a, true);  // stored only when the state asks for a sample
  a.host_f = h->host_f;
  a.host_ld = h->host_ld;
  a.out_z = h->out_z;
  a.out_ld = h->out_ld;
  // the pass count given here only sizes nothing: the kernel reads it from st
  CK(launch_gemm_tc((const uint16_t*)h->dh.p, (const uint16_t*)h->dl.p,
                    (const uint16_t*)h->wh.p, (const uint16_t*)h->wl.p, a, p.npad, p.kpad, 1,
                    p.bf16 ? 1 : 0, p.product_kernel, s));
  if (t) CK(cudaEventRecord(ev[3], s));  // the product kernel alone
  launch_sample_exact((const float*)h->drow.p, nullptr, (const int32_t*)h->icol.p, p.n, p.k,
                      p.kpad, p.npad, (const float*)h->smp.p, sample_stride(p),
                      sample_stride(p) / 2, (char*)h->smp.p + smp_scratch_off(p), st, dz, s);
  h->launches += 3;
  return IPT_OK;
}

// After the stream is synchronised: add this evaluation's event times.
void collect_timing(ipt_handle* h, int passes, Timing* tm, const cudaEvent_t* ev = nullptr,
                    int stage = -1) {
  if (!tm || !tm->on) return;
  if (!ev) ev = h->ev;
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess) tm->prepass_ms += a;
  if (passes == 0) return;
  const int slot = stage == IPT_PREC_F32C ? 2 : (passes == 3 ? 1 : 0);
  if (cudaEventElapsedTime(&b, ev[2], ev[3]) == cudaSuccess) tm->product_ms[slot] += b;
  tm->product_launches[slot] += 1;
}

void fill_result(const DevState& hs, const Timing& tm, int launches, ipt_result* out) {
  out->kernel_launches = launches;
  out->setup_ms = tm.setup_ms;
  out->finalize_ms = tm.finalize_ms;
  for (int i = 0; i < 2; ++i) {
    out->product_launches[i] = tm.product_launches[i];
    out->product_ms[i] = tm.product_ms[i];
  }
  out->acc_launches = tm.product_launches[2];
  out->acc_ms = tm.product_ms[2];
  out->rho_error = hs.e_rel;
  out->epilogue_operands = hs.epi_used;
  out->prepass_ms = tm.prepass_ms;
  out->status = hs.status;
  out->iterations = hs.iter;
  out->stage_iters[0] = hs.stage_iters[0];
  out->stage_iters[1] = hs.stage_iters[1];
  out->increment = hs.inc;
  out->rho = hs.rho;
  out->r0 = sqrt(hs.r0acc);
  out->rows_evaluated = hs.rows_eval;
  out->history_len = std::min(hs.iter, IPT_MAX_HISTORY);
  for (int i = 0; i < out->history_len; ++i) {
    out->hist_increment[i] = hs.hist_inc[i];
    out->hist_rho[i] = hs.hist_rho[i];
    out->hist_stage[i] = hs.hist_stage[i];
  }
}

ipt_status verify_fp64(ipt_handle* h, const Plan& p, const void* M, int64_t ldm, int m_dtype,
                       int zbuf, const double* lambda, double* rho64) {
  cudaStream_t s = h->s;
  const size_t nn = (size_t)p.npad * p.npad, kn = (size_t)p.kpad * p.npad;
  CK(ensure(h->m64, nn * 8));
  CK(ensure(h->z64, kn * 8));
  CK(ensure(h->racc, 8));
  launch_convert_m64(M, ldm, m_dtype, p.n, p.npad, (double*)h->m64.p, s);
  CK(cudaMemsetAsync(h->z64.p, 0, kn * 8, s));
  launch_copy_z(h->z[zbuf].p, p.f64 ? 1 : 0, p.npad, p.n, p.k, h->z64.p, p.npad, 1, s);
  CK(cudaMemsetAsync(h->racc.p, 0, 8, s));
  launch_residual_f64((const double*)h->m64.p, (const double*)h->z64.p, p.npad, lambda, p.n, p.k,
                      p.npad, p.kpad, (double*)h->racc.p, s);
  h->launches += 3;
  CK(cudaGetLastError());
  double r2 = 0.0, r0 = 0.0;
  CK(cudaMemcpyAsync(&r2, h->racc.p, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&r0, &dst(h)->r0acc, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *rho64 = r0 > 0.0 ? sqrt(r2) / sqrt(r0) : 0.0;
  return IPT_OK;
}

Plan make_plan(int64_t n, int64_t k, int prec, bool staged_bf16) {
  Plan p;
  p.n = (int)n;
  p.k = (int)k;
  p.npad = (int)round_up(n, kRowPad);
  p.kpad = (int)round_up(k, kColPad);
  p.prec = prec;
  p.f64 = prec == IPT_PREC_F64;
  p.tc = tensor_core(prec);
  p.bf16 = bf16_operands(prec, staged_bf16);
  p.dt = !p.f64;
  p.staged = prec == IPT_PREC_STAGED;
  return p;
}

// Unit errors of the product kinds, relative to ||Delta V|| (see k_control),
// for sums of length K = npad.  1-pass 16-bit: the operands' rounding (2^-11
// each for FP16, 2^-8 for BF16), taken as 2^-10 / 2^-7.  Split x3: the tensor
// core's FP32 accumulation, which drops low bits at each accumulate so its
// error grows with the K/16 accumulates of a pass: measured at n = 4096 and
// 8192 from 0.015 (K/16) 2^-24 (random-sign terms, the far K blocks first) to
// 0.66 (K/16) 2^-24 (the paper's U[0,1] family, whose sums grow coherently),
// taken at the upper end; for BF16 also the ~2^-16 of the split operands.
// FP32 SIMT: sequential FMA sums, 0.1-0.6 sqrt(K) 2^-24 measured, taken as
// 1.2.  Compensated FP32: one 32-long FP32 partial plus the pair's rounding.
// FP32 iterate arithmetic: 2^-23 of ||R0|| + ||Delta W||.
void set_error_model(ControlArgs& ca, const Plan& p) {
  const double K = (double)p.npad, u24 = ldexp(1.0, -24);
  ca.u_low = p.bf16 ? ldexp(1.0, -7) : ldexp(1.0, -10);
  ca.u_high = std::max(p.bf16 ? ldexp(1.0, -15) : ldexp(1.0, -20),
                       kSplitAccum * (K / 16.0) * u24);
  ca.u_f32 = 1.2 * sqrt(K) * u24;
  ca.u_acc = (0.6 * sqrt(32.0) + 2.0) * u24;
  ca.e_arith = p.f64 ? ldexp(1.0, -51) : ldexp(1.0, -23);
  ca.guard = 1;
}

// IPT-ACX (Alg. 3 in place of the Picard update of Alg. 1/2).  Buffer 0
// holds the extrapolated iterate z, buffers 1..3 hold f(z), f^2(z), f^3(z).
// An extrapolation of order p evaluates F at z (with Alg. 3's stopping test;
// d goes to the handle's d, so Lambda is z's) and at f(z) [, f^2(z)] (no
// test), then moves z in place.  Orders 3, 2, 3, 2, ...  One host
// synchronisation per extrapolation; every kernel returns at entry once the
// controller has stopped.
// Accelerated staged solves (p.acx_base): when the controller asks for it
// (want_acc), the next tested evaluation runs the compensated FP32 product,
// stores its P as the base product P_b and z is copied to buffer 4 as Z_b;
// later split products are of V = Z - Z_b.
ipt_status acx_loop(ipt_handle* h, const Plan& p, const ControlArgs& ca, const FirstEval& fe,
                    int max_iter, int sigma_global, Timing* tm, int start_iter = 0) {
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  const int split = (fe.stage == IPT_PREC_BF16X3 || fe.stage == IPT_PREC_FP16X3) ? 3 : 1;
  double* dinner = (double*)h->acx_d.p;
  CK(cudaMemsetAsync(h->acx_acc.p, 0, (size_t)p.kpad * 2 * 8, s));
  const size_t zbytes = (size_t)p.kpad * p.npad * (p.f64 ? 8 : 4);
  int done_evals = start_iter, base = -1;
  bool acc_next = false;
  double last_rho = 1.0;  // the last tested residual (sampling starts near tol)
  int stg_of[3] = {0, 0, 0}, passes_of[3] = {0, 0, 0};
  for (int step = 0; done_evals < max_iter; ++step) {
    const int order = (step % 2 == 0) ? 3 : 2;
    const int planned = std::min(order, max_iter - done_evals);
    for (int q = 0; q < planned; ++q) {
      int stg = fe.stage, passes = (done_evals + q == 0) ? fe.passes : (p.f64 ? 1 : split);
      int eb = base, rebase = 0;
      if (q == 0 && acc_next && p.acx_base) {
        stg = IPT_PREC_F32C;
        passes = 1;
        eb = -1;
        rebase = 1;
      }
      stg_of[q] = stg;
      passes_of[q] = passes;
      // tested tensor-core evaluations near tol sample their product error
      const int meas = (q == 0 && p.tc && passes > 0 && stg != IPT_PREC_F32C &&
                        last_rho <= 100.0 * ca.tol) ? 1 : 0;
      ControlArgs cq = ca;
      cq.acx = 1;
      cq.test = q == 0 ? 1 : 0;
      cq.host_base = eb;
      cq.host_rebase = rebase;
      cq.host_stage = stg;
      cq.host_passes = passes;
      cq.host_measure = meas;
      ipt_status v = evaluate(h, p, q, eb, stg, passes, rebase, tm, q + 1,
                              q == 0 ? nullptr : dinner + (size_t)(q - 1) * p.kpad,
                              h->evb + 4 * q, meas);
      if (v != IPT_OK) return v;
      launch_control(st, cq, s);
      h->launches += 1;
      if (rebase) {  // Z_b = z (buffer 0 is not moved before the extrapolation)
        CK(cudaMemcpyAsync(h->z[4].p, h->z[0].p, zbytes, cudaMemcpyDeviceToDevice, s));
        base = 4;
      }
    }
    if (planned == order) {
      launch_acx_combine(h->z[0].p, h->z[1].p, h->z[2].p, h->z[order == 3 ? 3 : 2].p,
                         p.f64 ? 1 : 0, order, p.n, p.k, p.npad, sigma_global,
                         (double*)h->acx_acc.p, (double*)h->acx_sigma.p, st, s);
      h->launches += 3;
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h->hst, st, kStateHead, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return IPT_CUDA_ERROR;
    if (step == 0 && start_iter == 0) {
      const ipt_status v = status_from_flags(h->hst->flags);
      if (v != IPT_OK) return v;
      if (tm && tm->on) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]) == cudaSuccess) tm->setup_ms = ms;
      }
    }
    const int ran = std::min(planned, h->hst->iter - done_evals);
    for (int q = 0; q < ran; ++q) collect_timing(h, passes_of[q], tm, h->evb + 4 * q, stg_of[q]);
    done_evals = h->hst->iter;
    if (h->hst->timeout) return IPT_DEVICE_TIMEOUT;
    if (h->hst->done) break;
    acc_next = p.acx_base && h->hst->want_acc;
    last_rho = h->hst->rho;
  }
  return IPT_OK;
}

// The Picard loop of a tensor-core solve without per-evaluation host work:
// the first evaluation as planned by the host, then evaluations with
// device-chosen operands, kDenseChunk per host synchronisation (every kernel
// returns at entry once the controller has stopped, so the evaluations
// enqueued past the stop cost only their launches).  When the controller
// chooses a compensated FP32 re-base, which the enqueued tensor-core kernels
// cannot run, it pauses them; the host then runs that evaluation itself and
// goes on.
ipt_status dense_chunked_loop(ipt_handle* h, const Plan& p, const ControlArgs& ca_in,
                              const FirstEval& fe, int max_iter, Timing* tm,
                              bool* handed_over = nullptr) {
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  const bool t = tm && tm->on;
  ControlArgs ca = ca_in;
  ca.pause_on_acc = 1;
  int done_evals = 0;
  bool first = true;
  auto sync_state = [&]() -> bool {
    return cudaGetLastError() == cudaSuccess &&
           cudaMemcpyAsync(h->hst, st, t ? sizeof(DevState) : kStateHead,
                           cudaMemcpyDeviceToHost, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
  };
  while (done_evals < max_iter) {
    const int nb = std::min(kDenseChunk, max_iter - done_evals);
    for (int q = 0; q < nb; ++q) {
      cudaEvent_t* ev = h->evb + 4 * q;
      const ipt_status v = (first && q == 0)
                               ? evaluate(h, p, 0, -1, fe.stage, fe.passes, fe.rebase, tm, -1,
                                          nullptr, ev)
                               : evaluate_dyn(h, p, tm, ev);
      if (v != IPT_OK) return v;
      launch_control(st, ca, s, true);
      h->launches += 1;
    }
    // with timing, the stage history tells each evaluation's pass count
    if (!sync_state()) return IPT_CUDA_ERROR;
    if (first) {
      const ipt_status fv = status_from_flags(h->hst->flags);
      if (fv != IPT_OK) return fv;
      if (t) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]) == cudaSuccess) tm->setup_ms = ms;
      }
    }
    first = false;
    if (t) {
      const int ran = std::min(nb, h->hst->iter - done_evals);
      for (int q = 0; q < ran; ++q) {
        const int e = done_evals + q;
        const int stg = e < IPT_MAX_HISTORY ? h->hst->hist_stage[e] : p.prec;
        const int passes =
            stg < 0 ? 0 : ((stg == IPT_PREC_BF16X3 || stg == IPT_PREC_FP16X3) ? 3 : 1);
        collect_timing(h, passes, tm, h->evb + 4 * q);
      }
    }
    done_evals = h->hst->iter;
    if (h->hst->timeout) return IPT_DEVICE_TIMEOUT;
    if (h->hst->done) break;
    if (h->hst->pause == 2 && handed_over) {  // the acceleration continues the solve
      *handed_over = true;
      CK(cudaMemsetAsync(&st->pause, 0, sizeof(int), s));
      CK(cudaMemsetAsync(&st->split_ready, 0, sizeof(int), s));  // its products' own operands
      return IPT_OK;
    }
    if (h->hst->pause) {
      CK(cudaMemsetAsync(&st->pause, 0, sizeof(int), s));
      const int stg = h->hst->stage;
      const ipt_status v = evaluate(h, p, h->hst->cur, h->hst->base, stg, h->hst->passes,
                                    h->hst->rebase, tm, -1, nullptr, h->ev);
      if (v != IPT_OK) return v;
      launch_control(st, ca, s, true);
      h->launches += 1;
      if (!sync_state()) return IPT_CUDA_ERROR;
      collect_timing(h, 1, tm, h->ev, stg);
      done_evals = h->hst->iter;
      if (h->hst->timeout) return IPT_DEVICE_TIMEOUT;
      if (h->hst->done) break;
    }
  }
  return IPT_OK;
}

// Anderson mixing (IPT_ACCEL_ANDERSON), or with `mix_model` the learned damping
// and mixing (IPT_ACCEL_MIXING, k_mix.cu) on the same buffers.  Buffers: zc holds the iterate under
// test, (zp, gp) the previous iterate and its map value, fr receives this
// evaluation's map value.  The first step is a Picard step, so z_1 = g_0 stays
// where g_0 was written (zc = gp); later steps write z_{t+1} over z_{t-1}.  One
// host synchronisation per evaluation.  Accelerated staged solves re-base as in
// acx_loop (Z_b in buffer 4).
ipt_status anderson_loop(ipt_handle* h, const Plan& p, const ControlArgs& ca,
                         const FirstEval& fe, int max_iter, Timing* tm,
                         const void* mix_model = nullptr, int start_iter = 0) {
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  const int split = (fe.stage == IPT_PREC_BF16X3 || fe.stage == IPT_PREC_FP16X3) ? 3 : 1;
  double* acc = (double*)h->acx_acc.p;
  double* gamma = (double*)h->acx_sigma.p;
  AndState* as = reinterpret_cast<AndState*>(h->acx_d.p);
  CK(cudaMemsetAsync(acc, 0, (size_t)p.kpad * 2 * 8, s));
  CK(cudaMemsetAsync(as, 0, sizeof(AndState), s));
  // learned mixing scratch (see mix_bytes)
  double* macc = mix_model ? (double*)h->mix.p : nullptr;
  double* hlam = macc ? macc + (size_t)4 * p.kpad : nullptr;
  float* hinc = macc ? (float*)(hlam + (size_t)3 * p.kpad) : nullptr;
  float* X = hinc ? hinc + (size_t)3 * p.kpad : nullptr;
  float* ag = X ? X + (size_t)kMixInputs * p.kpad : nullptr;
  DampState* ms = ag ? reinterpret_cast<DampState*>(ag + (size_t)2 * p.kpad) : nullptr;
  if (mix_model) CK(cudaMemsetAsync(h->mix.p, 0, mix_bytes(p.kpad), s));
  int zc = 0, zp = -1, gp = -1, fr = 1;
  const size_t zbytes = (size_t)p.kpad * p.npad * (p.f64 ? 8 : 4);
  int base = -1;
  bool acc_next = false;
  double last_rho = 1.0;
  for (int it = 0; it < max_iter - start_iter; ++it) {
    int stg = fe.stage, passes = (it == 0 && start_iter == 0) ? fe.passes : (p.f64 ? 1 : split);
    int eb = base, rebase = 0;
    if (acc_next) {
      stg = IPT_PREC_F32C;
      passes = 1;
      eb = -1;
      rebase = 1;
    }
    ControlArgs cq = ca;
    cq.acx = 1;
    cq.next_cur = it == 0 ? fr : zp;  // where the next iterate will be
    const int meas =
        (p.tc && passes > 0 && stg != IPT_PREC_F32C && last_rho <= 100.0 * ca.tol) ? 1 : 0;
    cq.host_base = eb;
    cq.host_rebase = rebase;
    cq.host_stage = stg;
    cq.host_passes = passes;
    cq.host_measure = meas;
    ipt_status v = evaluate(h, p, zc, eb, stg, passes, rebase, tm, fr, nullptr, nullptr, meas);
    if (v != IPT_OK) return v;
    launch_control(st, cq, s);
    if (rebase) {
      CK(cudaMemcpyAsync(h->z[4].p, h->z[zc].p, zbytes, cudaMemcpyDeviceToDevice, s));
      base = 4;
    }
    if (mix_model) {
      CK(launch_mix_step(h->z[zc].p, h->z[fr].p, it ? h->z[zp].p : nullptr,
                         it ? h->z[gp].p : nullptr, it ? h->z[zp].p : nullptr, p.f64 ? 1 : 0,
                         p.n, p.k, p.npad, (const double*)h->theta.p, (const int32_t*)h->icol.p,
                         (const double*)h->d.p, mix_model, macc, hinc, hlam, X, ag, ms, st, s));
      h->launches += it == 0 ? 4 : 5;
    } else {
      CK(launch_anderson_step(h->z[zc].p, h->z[fr].p, it ? h->z[zp].p : nullptr,
                              it ? h->z[gp].p : nullptr, it ? h->z[zp].p : nullptr,
                              p.f64 ? 1 : 0, p.n, p.k, p.npad, acc, gamma, as, st, it == 0, s));
      h->launches += it == 0 ? 3 : 5;
    }
    if (cudaMemcpyAsync(h->hst, st, kStateHead, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return IPT_CUDA_ERROR;
    if (it == 0 && start_iter == 0) {
      const ipt_status fv = status_from_flags(h->hst->flags);
      if (fv != IPT_OK) return fv;
      if (tm && tm->on) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]) == cudaSuccess) tm->setup_ms = ms;
      }
    }
    collect_timing(h, passes, tm, nullptr, stg);
    if (h->hst->timeout) return IPT_DEVICE_TIMEOUT;
    if (h->hst->done) break;
    acc_next = p.acx_base && h->hst->want_acc;
    last_rho = h->hst->rho;
    if (it == 0) {
      zp = zc;
      gp = fr;
      zc = fr;
    } else {
      const int ozc = zc, ozp = zp;
      zc = ozp;
      zp = ozc;
      gp = fr;
    }
    fr = 0;  // the buffer holding none of zc, zp, gp
    while (fr == zc || fr == zp || fr == gp) ++fr;
  }
  return IPT_OK;
}

ipt_status solve_dense(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                       const double* theta, int64_t k, const int32_t* cols, double tol,
                       int max_iter, const ipt_options* opt_in, double* lambda, void* Z,
                       int64_t ldz, int z_dtype, ipt_result* out,
                       const HostOut* hz = nullptr) {
  if (!out) return IPT_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->rho_fp64 = -1.0;
  ipt_options opt;
  ipt_options_default(&opt);
  if (opt_in) opt = *opt_in;
  ipt_status v = check_dense_args(h, n, M, ldm, m_dtype, k, opt.precision, ldz, z_dtype);
  if (v == IPT_OK && (!lambda || !Z || !(tol >= 0.0) || max_iter < 1 ||
                      (opt.stop != IPT_STOP_INCREMENT && opt.stop != IPT_STOP_RESIDUAL) ||
                      opt.product_kernel < IPT_PRODUCT_AUTO ||
                      opt.product_kernel > IPT_PRODUCT_PAIR ||
                      (opt.accel != IPT_ACCEL_NONE && opt.accel != IPT_ACCEL_ACX &&
                       opt.accel != IPT_ACCEL_DAMPED && opt.accel != IPT_ACCEL_ANDERSON &&
                       opt.accel != IPT_ACCEL_MIXING) ||
                      ((opt.accel == IPT_ACCEL_DAMPED || opt.accel == IPT_ACCEL_MIXING) &&
                       !opt.damping_model) ||
                      (opt.acx_sigma != 0 && opt.acx_sigma != 1)))
    v = IPT_INVALID_ARG;
  if (v != IPT_OK) {
    out->status = v;
    return v;
  }
  DeviceGuard g(h->dev);
  const auto t_start = std::chrono::steady_clock::now();
  h->launches = 0;
  Timing tm;
  tm.on = opt.record_timing != 0;
  if (tm.on && ensure_events(h) != IPT_OK) {
    out->status = IPT_CUDA_ERROR;
    return IPT_CUDA_ERROR;
  }
  const bool acx = opt.accel == IPT_ACCEL_ACX;
  const bool damped = opt.accel == IPT_ACCEL_DAMPED;
  const bool mixing = opt.accel == IPT_ACCEL_MIXING;
  const bool anderson = opt.accel == IPT_ACCEL_ANDERSON || mixing;
  // ACX and Anderson mixing move the iterate by extrapolation, outside the
  // staged schedule's step model: a staged request runs the split products,
  // first of W = Z - E and, once their error model asks for it, of Z minus a
  // base stored by one compensated FP32 evaluation.  (Damped steps stay inside
  // the staged schedule with a step bound of 2 increments.)
  const bool accel_staged = (acx || anderson) && opt.precision == IPT_PREC_STAGED;
  // Staged accelerated solves begin as the staged Picard solve (device-chosen
  // operands, no per-evaluation host work) and hand over to the acceleration
  // only once the residual contracts slowly: on problems where Picard converges
  // fast they cost what the staged solve costs.  (Not with host buffers.)
  const bool handover = (accel_staged || damped) && opt.precision == IPT_PREC_STAGED && !hz &&
                        !opt.z0;
  const int prec = accel_staged ? (opt.staged_bf16 ? IPT_PREC_BF16X3 : IPT_PREC_FP16X3)
                                : opt.precision;
  Plan p = make_plan(n, k, prec, opt.staged_bf16 != 0);
  p.epi_operand = p.staged && p.tc && opt.epilogue_operand != 0;
  bool out_direct = false;  // the returned iterate may be stored into Z by its product
  p.product_kernel = opt.product_kernel;
  p.acx = acx || anderson;  // four iterate buffers and the per-column scratch
  p.acx_base = accel_staged;
  p.damped = damped;
  p.mixing = mixing;
  const int low = p.bf16 ? IPT_PREC_BF16 : IPT_PREC_FP16;
  const int high = p.bf16 ? IPT_PREC_BF16X3 : IPT_PREC_FP16X3;
  // First evaluation: product-free at Z = E (FP32 / tensor-core paths), else
  // a product; a staged solve from a warm start begins with a split product
  // and re-bases on it.
  FirstEval fe;
  fe.stage = prec == IPT_PREC_STAGED ? (opt.z0 ? high : low) : prec;
  fe.passes = (!p.f64 && !opt.z0)
                  ? 0
                  : ((fe.stage == IPT_PREC_BF16X3 || fe.stage == IPT_PREC_FP16X3) ? 3 : 1);
  fe.rebase = (p.staged && opt.z0) ? 1 : 0;
  fe.accurate = 1;
  fe.defer_e = !acx && !damped && !anderson && !hz;  // the update / copy-out reads z = E
  // the staged Picard phase of a hand-over solve: its own plan and first stage
  Plan pst = p;
  pst.staged = true;
  pst.prec = IPT_PREC_STAGED;
  pst.epi_operand = p.tc && opt.epilogue_operand != 0;
  FirstEval fe_run = fe;
  if (handover) {
    fe_run.stage = low;
    fe_run.passes = 0;
    fe_run.rebase = 0;
  }
  v = alloc_dense(h, p);
  if (v == IPT_OK && handover) v = alloc_dense(h, pst);
  if (v == IPT_OK) {
    if (tm.on) cudaEventRecord(h->ev[4], h->s);
    v = setup_dense(h, p, M, ldm, m_dtype, theta, cols, opt.z0, ldz, z_dtype, true, fe_run,
                    false);
    if (tm.on) cudaEventRecord(h->ev[5], h->s);
  }
  if (v != IPT_OK) {
    out->status = v;
    return v;
  }
  ControlArgs ca;
  ca.tol = tol;
  ca.diverge_bound = opt.diverge_bound;
  ca.stage_switch = opt.stage_switch;
  ca.max_iter = max_iter;
  ca.stop = opt.stop;
  ca.mode = prec;
  ca.k = (int)k;
  ca.low_stage = low;
  ca.high_stage = high;
  set_error_model(ca, p);
  ca.escalate = p.staged ? 1 : 0;
  ca.accel_staged = accel_staged ? 1 : 0;
  ca.smp_rows = p.tc ? sample_rows(p) : 0;
  ca.n_rows = p.n;
  // fixed-precision tensor-core Picard solves sample the product error of the
  // evaluations that may end the solve
  ca.measure_below = (p.tc && !p.staged && !acx && !anderson) ? 3.0 * tol : 0.0;
  cudaStream_t s = h->s;
  int cur = 0, base = -1, stage = fe.stage, passes = fe.passes, rebase = fe.rebase;
  int start = 0;  // evaluations done before the loop below (hand-over)
  bool handed_over = false;
  if (handover) {
    ControlArgs cst = ca;
    cst.mode = IPT_PREC_STAGED;
    cst.escalate = 1;
    cst.accel_staged = 0;
    cst.measure_below = 0.0;
    cst.slow_ratio = kHandoverRatio;
    v = dense_chunked_loop(h, pst, cst, fe_run, max_iter, &tm, &handed_over);
    if (v == IPT_OK && handed_over) {
      start = h->hst->iter;
      if (acx || anderson) {
        // the accelerations keep their iterate in buffer 0
        const int c = h->hst->cur;
        if (c != 0)
          CK(cudaMemcpyAsync(h->z[0].p, h->z[c].p, (size_t)p.kpad * p.npad * (p.f64 ? 8 : 4),
                             cudaMemcpyDeviceToDevice, s));
        h->hinit->cur = 0;
        CK(cudaMemcpyAsync(&dst(h)->cur, &h->hinit->cur, sizeof(int), cudaMemcpyHostToDevice,
                           s));
      } else {
        cur = h->hst->cur;
        base = h->hst->base;
        stage = h->hst->stage;
        passes = h->hst->passes;
        rebase = h->hst->rebase;
      }
    }
  }
  FirstEval fe_acc = fe;  // after a hand-over the accelerations start with a product
  if (handed_over) fe_acc.passes = (fe.stage == IPT_PREC_BF16X3 || fe.stage == IPT_PREC_FP16X3)
                                       ? 3 : 1;
  if (v != IPT_OK || (handover && !handed_over)) {
    max_iter = 0;  // solved (or failed) in the staged phase
  } else if (acx) {
    v = acx_loop(h, p, ca, fe_acc, max_iter, opt.acx_sigma, &tm, start);
    max_iter = 0;  // the Picard loop below does not run
  } else if (anderson) {
    v = anderson_loop(h, p, ca, fe_acc, max_iter, &tm, mixing ? opt.damping_model : nullptr,
                      start);
    max_iter = 0;
  } else if (p.tc && !damped && !hz) {
    // a staged Picard solve into an FP32 Z: the product that forms the
    // predicted result stores it into Z as well (no copy after the loop then)
    struct OutClear {
      ipt_handle* h;
      ~OutClear() { h->out_z = nullptr; }
    } out_clear{h};
    ControlArgs cc = ca;
    if (p.staged && !p.f64 && z_dtype == IPT_DTYPE_F32) {
      h->out_z = static_cast<float*>(Z);
      h->out_ld = ldz;
      cc.out_pred = 1;
      out_direct = true;
    }
    v = dense_chunked_loop(h, p, cc, fe, max_iter, &tm);
    max_iter = 0;
  }
  // learned damping: history, features, alphas and the damped next iterate,
  // formed in F's buffer after each evaluation that does not stop the solve
  double* dacc = nullptr;
  double* hlam = nullptr;
  float *hinc = nullptr, *X = nullptr, *alpha = nullptr;
  DampState* ds = nullptr;
  if (damped && max_iter > 0) {
    ca.step_scale = 2.0;
    // layout: lam history (3 kpad FP64), inc history (3 kpad), features
    // (6 kpad), alphas (kpad), state (kpad is a multiple of 256: all aligned)
    dacc = (double*)h->acx_acc.p;
    hlam = (double*)h->damp.p;
    hinc = (float*)(hlam + (size_t)3 * p.kpad);
    X = hinc + (size_t)3 * p.kpad;
    alpha = X + (size_t)6 * p.kpad;
    ds = reinterpret_cast<DampState*>(alpha + p.kpad);
    CK(cudaMemsetAsync(h->damp.p, 0, (size_t)p.kpad * (3 * 8 + 3 * 4 + 6 * 4 + 4) + 64, s));
    CK(cudaMemsetAsync(dacc, 0, (size_t)p.kpad * 2 * 8, s));
  }
  const size_t zes = p.f64 ? 8 : 4;
  // host output: the iterate under test is copied out beside its evaluation
  // when that evaluation is predicted to pass the test (test value times the
  // last contraction below tol, and a product accurate enough to stop on);
  // otherwise the returned iterate is copied after the loop
  // With the host output mapped into the device's address space, an evaluation
  // whose F is predicted to be the returned iterate (the test two evaluations on
  // passes: test value times the last contraction squared below tol) stores F
  // there from the product's epilogue, during the product.
  bool likely_final = false, write_next = false;
  int copied_it = -1, host_written_it = -1;
  struct HostFClear {  // never left set for a later launch, whatever the exit
    ipt_handle* h;
    ~HostFClear() { h->host_f = nullptr; }
  } host_f_clear{h};
  cudaEvent_t copy_in_flight = nullptr;
  double prev_test = -1.0;
  for (int it = start; it < max_iter; ++it) {
    if (hz && likely_final && host_written_it == it - 1) likely_final = false;  // on the host
    if (hz && likely_final) {
      // the output buffer of this evaluation must not still be copied out
      const int nxt = free_buffer(cur, base);
      if (h->zcopied[nxt]) CK(cudaStreamWaitEvent(s, h->zcopied[nxt], 0));
      CK(cudaEventRecord(h->zready, s));
      CK(cudaStreamWaitEvent(h->cs, h->zready, 0));
      CK(cudaMemcpy2DAsync(hz->Z, (size_t)hz->ldz * zes, h->z[cur].p, (size_t)p.npad * zes,
                           (size_t)p.n * zes, (size_t)p.k, cudaMemcpyDeviceToHost, h->cs));
      CK(cudaEventRecord(h->zcopied[cur], h->cs));
      copy_in_flight = h->zcopied[cur];
      copied_it = it;
    }
    // this evaluation's tensor-core epilogue writes F to the host output: after
    // any copy into the same buffer has finished
    const bool host_write = hz && hz->Zdev && write_next && p.tc && passes > 0 &&
                            stage != IPT_PREC_F32 && stage != IPT_PREC_F32C &&
                            stage != IPT_PREC_F64;
    if (host_write) {
      if (copy_in_flight) CK(cudaStreamWaitEvent(s, copy_in_flight, 0));
      h->host_f = (float*)hz->Zdev;
      h->host_ld = hz->ldz;
      host_written_it = it;
    }
    const int fbuf = free_buffer(cur, base);  // where this evaluation writes F
    // a staged Picard product runs as the device-chosen evaluation (the state
    // holds the same cur, base and pass count), so that its operand may come
    // from the previous product's epilogue as in the chunked loop
    const bool dyn_eval = p.epi_operand && !damped && it > 0 && passes > 0 &&
                          stage != IPT_PREC_F32 && stage != IPT_PREC_F32C;
    v = dyn_eval ? evaluate_dyn(h, p, &tm, h->ev)
                 : evaluate(h, p, cur, base, stage, passes, rebase, &tm, -1, nullptr, nullptr,
                            it > 0 && p.tc ? h->hst->measure : 0);
    h->host_f = nullptr;
    if (v != IPT_OK) break;
    launch_control(dst(h), ca, s);
    h->launches += 1;
    if (damped) {
      CK(launch_damp_step(h->z[cur].p, h->z[fbuf].p, p.f64 ? 1 : 0, p.n, p.k, p.npad,
                          (const double*)h->theta.p, (const int32_t*)h->icol.p,
                          (const double*)h->d.p, opt.damping_model, dacc, hinc, hlam, X, alpha,
                          ds, dst(h), s));
      h->launches += 5;
    }
    if (cudaMemcpyAsync(h->hst, dst(h), kStateHead, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      v = IPT_CUDA_ERROR;
      break;
    }
    if (it == 0) {
      // validation flags of the setup kernels, before any output is written
      v = status_from_flags(h->hst->flags);
      if (v != IPT_OK) break;
      if (tm.on) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]) == cudaSuccess) tm.setup_ms = ms;
      }
    }
    collect_timing(h, passes, &tm);
    if (h->hst->timeout) {
      v = IPT_DEVICE_TIMEOUT;
      break;
    }
    if (h->hst->done) break;
    cur = h->hst->cur;
    base = h->hst->base;
    stage = h->hst->stage;
    passes = h->hst->passes;
    rebase = h->hst->rebase;
    if (hz) {
      const double test = opt.stop == IPT_STOP_INCREMENT ? h->hst->inc : h->hst->rho;
      const double q = prev_test > 0.0 ? std::min(test / prev_test, 1.0) : 1.0;
      likely_final = (!p.staged || h->hst->accurate) && test * q <= tol;
      write_next = !likely_final && test * q * q <= tol;
      prev_test = test;
    }
  }
  if (v != IPT_OK) {
    out->status = v;
    return v;
  }
  DevState hs;
  if (cudaMemcpyAsync(&hs, dst(h), sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    out->status = IPT_CUDA_ERROR;
    return IPT_CUDA_ERROR;
  }
  const int ans = hs.answer;
  if (tm.on) cudaEventRecord(h->ev[6], s);
  // buffer 0 holds E only while no evaluation has written into it: the solve
  // stopped at its first evaluation
  if (ans == 0 && h->e_pending && hs.iter == 1) {
    launch_init_z(nullptr, 0, 0, (const int32_t*)h->icol.p, p.n, p.k, p.npad, p.kpad, h->z[0].p,
                  p.f64 ? 1 : 0, dst(h), s);
    h->e_pending = false;
    h->launches += 1;
  }
  launch_lambda((const double*)h->theta.p, (const int32_t*)h->icol.p, (const double*)h->d.p,
                p.k, lambda, s);
  h->launches += 1;
  if (hz) {
    if (copied_it != (int)hs.iter - 1 &&
        !(host_written_it >= 0 && host_written_it == (int)hs.iter - 2)) {
      // the returned iterate was not copied out beside its evaluation, nor
      // written out by the epilogue of the evaluation that formed it
      CK(cudaStreamSynchronize(h->cs));
      CK(cudaMemcpy2DAsync(hz->Z, (size_t)hz->ldz * zes, h->z[ans].p, (size_t)p.npad * zes,
                           (size_t)p.n * zes, (size_t)p.k, cudaMemcpyDeviceToHost, s));
    } else {
      CK(cudaStreamSynchronize(h->cs));
    }
  } else if (!(out_direct && hs.out_iter >= 0 && hs.out_iter == (int)hs.iter - 2)) {
    // (else the evaluation that formed the returned iterate stored it into Z)
    launch_copy_z(h->z[ans].p, p.f64 ? 1 : 0, p.npad, p.n, p.k, Z, ldz,
                  z_dtype == IPT_DTYPE_F64 ? 1 : 0, s);
    h->launches += 1;
  }
  if (tm.on) cudaEventRecord(h->ev[7], s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    out->status = IPT_CUDA_ERROR;
    return IPT_CUDA_ERROR;
  }
  if (tm.on) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[6], h->ev[7]) == cudaSuccess) tm.finalize_ms = ms;
  }
  fill_result(hs, tm, h->launches, out);
  out->wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (opt.verify_fp64) {
    v = verify_fp64(h, p, M, ldm, m_dtype, ans, lambda, &out->rho_fp64);
    if (v != IPT_OK) {
      out->status = v;
      return v;
    }
  }
  return (ipt_status)out->status;
}

}  // namespace

extern "C" {

void ipt_options_default(ipt_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = IPT_PREC_STAGED;
  opt->stop = IPT_STOP_RESIDUAL;
  opt->diverge_bound = 1e8;
  opt->stage_switch = 0.1;
  opt->staged_bf16 = 0;
  opt->verify_fp64 = 0;
  opt->record_timing = 0;
  opt->z0 = nullptr;
  opt->product_kernel = IPT_PRODUCT_AUTO;
  opt->csr_window = 1;
  opt->epilogue_operand = 1;
}

const char* ipt_status_string(int status) {
  switch (status) {
    case IPT_OK: return "IPT_OK";
    case IPT_MAXITER: return "IPT_MAXITER";
    case IPT_DIVERGED: return "IPT_DIVERGED";
    case IPT_DEGENERATE_THETA: return "IPT_DEGENERATE_THETA";
    case IPT_INVALID_ARG: return "IPT_INVALID_ARG";
    case IPT_CUDA_ERROR: return "IPT_CUDA_ERROR";
    case IPT_DEVICE_TIMEOUT: return "IPT_DEVICE_TIMEOUT";
    case IPT_UNSUPPORTED: return "IPT_UNSUPPORTED";
    case IPT_INACCURATE: return "IPT_INACCURATE";
    default: return "IPT_UNKNOWN_STATUS";
  }
}

ipt_status ipt_create(ipt_handle** h, void* stream) {
  if (!h) return IPT_INVALID_ARG;
  *h = nullptr;
  ipt_handle* x = new ipt_handle();
  x->s = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&x->dev) != cudaSuccess ||
      cudaMallocHost((void**)&x->hst, sizeof(DevState)) != cudaSuccess ||
      cudaMallocHost((void**)&x->hinit, sizeof(DevState)) != cudaSuccess) {
    if (x->hst) cudaFreeHost(x->hst);
    delete x;
    return IPT_CUDA_ERROR;
  }
  *h = x;
  return IPT_OK;
}

ipt_status ipt_destroy(ipt_handle* h) {
  if (!h) return IPT_OK;
  DeviceGuard g(h->dev);
  Buf* all[] = {&h->drow, &h->dt, &h->dh, &h->dl, &h->z[0], &h->z[1], &h->z[2], &h->z[3],
                &h->acx_d, &h->acx_acc, &h->acx_sigma, &h->damp, &h->bmeta, &h->bscratch,
                &h->pbuf, &h->z[4], &h->smp, &h->mix, &h->wh2, &h->wl2, &h->dpart,
                &h->wh, &h->wl,
                &h->rinv, &h->sinv, &h->theta, &h->thh, &h->thl, &h->icol, &h->count,
                &h->r0part, &h->delta, &h->cpart,
                &h->d, &h->st, &h->m64, &h->z64, &h->racc, &h->hM, &h->hTheta, &h->hCols,
                &h->hLam, &h->hZ};
  for (Buf* b : all)
    if (b->p) cudaFree(b->p);
  for (int i = 0; i < 8; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  for (int i = 0; i < 4 * kEvbSlots; ++i)
    if (h->evb[i]) cudaEventDestroy(h->evb[i]);
  if (h->zready) cudaEventDestroy(h->zready);
  for (int b = 0; b < 3; ++b)
    if (h->zcopied[b]) cudaEventDestroy(h->zcopied[b]);
  if (h->cs) cudaStreamDestroy(h->cs);
  if (h->hst) cudaFreeHost(h->hst);
  if (h->hinit) cudaFreeHost(h->hinit);
  if (h->hmeta) cudaFreeHost(h->hmeta);
  if (h->hstat) cudaFreeHost(h->hstat);
  if (h->bexec) cudaGraphExecDestroy(h->bexec);
  if (h->bgraph) cudaGraphDestroy(h->bgraph);
  if (h->gs) cudaStreamDestroy(h->gs);
  delete h;
  return IPT_OK;
}

ipt_status ipt_solve_dense(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                           const double* theta, int64_t k, const int32_t* cols, double tol,
                           int max_iter, const ipt_options* opt, double* lambda, void* Z,
                           int64_t ldz, int z_dtype, ipt_result* out) {
  return solve_dense(h, n, M, ldm, m_dtype, theta, k, cols, tol, max_iter, opt, lambda, Z, ldz,
                     z_dtype, out);
}

ipt_status ipt_solve_dense_host(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                                const double* theta, int64_t k, const int32_t* cols, double tol,
                                int max_iter, const ipt_options* opt, double* lambda, void* Z,
                                int64_t ldz, int z_dtype, ipt_result* out) {
  if (!out) return IPT_INVALID_ARG;
  ipt_options o;
  ipt_options_default(&o);
  if (opt) o = *opt;
  ipt_status v = check_dense_args(h, n, M, ldm, m_dtype, k, o.precision, ldz, z_dtype);
  if (v != IPT_OK || !lambda || !Z || o.z0) {
    memset(out, 0, sizeof(*out));
    out->status = v != IPT_OK ? v : IPT_INVALID_ARG;
    return (ipt_status)out->status;
  }
  DeviceGuard g(h->dev);
  cudaStream_t s = h->s;
  const size_t em = m_dtype == IPT_DTYPE_F64 ? 8 : 4, ez = z_dtype == IPT_DTYPE_F64 ? 8 : 4;
  // Pinned (mapped) host buffers are used in place: the setup reads M over the
  // host link while it forms Delta (no staging copy), and the product epilogue
  // of the evaluation predicted to form the returned iterate stores it into Z.
  // Pageable buffers go through device copies.
  auto mapped = [](const void* ptr) -> void* {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
  };
  const void* Mdev = mapped(M);
  CK(ensure(h->hLam, (size_t)k * 8));
  CK(ensure(h->hZ, (size_t)n * k * ez));
  if (!Mdev) {
    CK(ensure(h->hM, (size_t)n * n * em));
    CK(cudaMemcpy2DAsync(h->hM.p, n * em, M, ldm * em, n * em, n, cudaMemcpyHostToDevice, s));
  }
  const bool iter_f64 = o.precision == IPT_PREC_F64;
  const bool direct = o.accel == IPT_ACCEL_NONE && (z_dtype == IPT_DTYPE_F64) == iter_f64;
  HostOut ho;
  if (direct) {
    if (!h->cs) CK(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
    if (!h->zready) CK(cudaEventCreateWithFlags(&h->zready, cudaEventDisableTiming));
    for (int b = 0; b < 3; ++b)
      if (!h->zcopied[b]) CK(cudaEventCreateWithFlags(&h->zcopied[b], cudaEventDisableTiming));
  }
  const double* dth = nullptr;
  const int32_t* dcols = nullptr;
  if (theta) {
    CK(ensure(h->hTheta, (size_t)n * 8));
    CK(cudaMemcpyAsync(h->hTheta.p, theta, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    dth = (const double*)h->hTheta.p;
  }
  if (cols) {
    CK(ensure(h->hCols, (size_t)k * 4));
    CK(cudaMemcpyAsync(h->hCols.p, cols, (size_t)k * 4, cudaMemcpyHostToDevice, s));
    dcols = (const int32_t*)h->hCols.p;
  }
  // the iterate is copied straight from the solver's buffers to Z when its
  // dtype is Z's (FP32 iterate unless the FP64 product is asked for) and the
  // Picard loop runs; otherwise through a device copy
  if (direct) {
    ho.Z = Z;
    ho.ldz = ldz;
    ho.Zdev = mapped(Z);
  }
  v = solve_dense(h, n, Mdev ? Mdev : h->hM.p, Mdev ? ldm : n, m_dtype, dth, k, dcols, tol,
                  max_iter, &o, (double*)h->hLam.p, h->hZ.p, n, z_dtype, out,
                  direct ? &ho : nullptr);
  if (v == IPT_OK || v == IPT_MAXITER || v == IPT_DIVERGED || v == IPT_INACCURATE) {
    CK(cudaMemcpyAsync(lambda, h->hLam.p, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    if (!direct)
      CK(cudaMemcpy2DAsync(Z, ldz * ez, h->hZ.p, n * ez, n * ez, k, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (direct && h->cs) cudaStreamSynchronize(h->cs);  // no copy out may outlive the call
  return v;
}

ipt_status ipt_step_dense(ipt_handle* h, int64_t n, const void* M, int64_t ldm, int m_dtype,
                          const double* theta, int64_t k, const int32_t* cols, int precision,
                          const void* Zin, void* Fout, int64_t ldz, int z_dtype, double* lambda,
                          double* norms) {
  ipt_status v = check_dense_args(h, n, M, ldm, m_dtype, k, precision, ldz, z_dtype);
  if (v != IPT_OK) return v;
  if (precision == IPT_PREC_STAGED || !Zin || !Fout || !lambda) return IPT_INVALID_ARG;
  DeviceGuard g(h->dev);
  const Plan p = make_plan(n, k, precision, false);
  v = alloc_dense(h, p);
  if (v != IPT_OK) return v;
  FirstEval fe;
  fe.stage = precision;
  fe.passes = (precision == IPT_PREC_BF16X3 || precision == IPT_PREC_FP16X3) ? 3 : 1;
  fe.rebase = 0;
  fe.accurate = 1;
  v = setup_dense(h, p, M, ldm, m_dtype, theta, cols, Zin, ldz, z_dtype, false, fe, true);
  if (v != IPT_OK) return v;
  v = evaluate(h, p, 0, -1, precision, fe.passes, 0, nullptr);
  if (v != IPT_OK) return v;
  cudaStream_t s = h->s;
  CK(cudaMemcpyAsync(h->hst, dst(h), kStateHead, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  v = status_from_flags(h->hst->flags);  // theta_j == theta_{cols[c]} is found in the epilogue
  if (v != IPT_OK) return v;
  launch_lambda((const double*)h->theta.p, (const int32_t*)h->icol.p, (const double*)h->d.p,
                p.k, lambda, s);
  launch_copy_z(h->z[1].p, p.f64 ? 1 : 0, p.npad, p.n, p.k, Fout, ldz,
                z_dtype == IPT_DTYPE_F64 ? 1 : 0, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->hst, dst(h), kStateHead, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h->hst->timeout) return IPT_DEVICE_TIMEOUT;
  if (norms) {
    norms[0] = sqrt(h->hst->acc_inc2);
    norms[1] = sqrt(h->hst->acc_z2);
    norms[2] = sqrt(h->hst->acc_r2);
  }
  return IPT_OK;
}

ipt_status ipt_solve_csr(ipt_handle* h, int64_t n, int64_t nnz, const int32_t* rowptr,
                         const int32_t* colind, const void* vals, int v_dtype,
                         const double* theta, int64_t k, const int32_t* cols, double tol,
                         int max_iter, const ipt_options* opt_in, double* lambda, void* Z,
                         int64_t ldz, int z_dtype, ipt_result* out) {
  if (!out) return IPT_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->rho_fp64 = -1.0;
  ipt_options opt;
  ipt_options_default(&opt);
  if (opt_in) opt = *opt_in;
  ipt_status v = IPT_OK;
  if (!h || !rowptr || !vals || (nnz > 0 && !colind) || !lambda || !Z || n < 1 ||
      n > (int64_t)1 << 30 || nnz < 0 || nnz >= ((int64_t)1 << 31) || k < 1 || k > n ||
      ldz < n || !(tol >= 0.0) || max_iter < 1 ||
      (v_dtype != IPT_DTYPE_F64 && v_dtype != IPT_DTYPE_F32) ||
      (z_dtype != IPT_DTYPE_F64 && z_dtype != IPT_DTYPE_F32) ||
      (opt.stop != IPT_STOP_INCREMENT && opt.stop != IPT_STOP_RESIDUAL) || opt.z0 ||
      opt.accel < IPT_ACCEL_NONE || opt.accel > IPT_ACCEL_ANDERSON ||
      (opt.acx_sigma != 0 && opt.acx_sigma != 1))
    v = IPT_INVALID_ARG;
  int prec = opt.precision == IPT_PREC_STAGED ? IPT_PREC_F32 : opt.precision;
  if (v == IPT_OK && prec != IPT_PREC_F32 && prec != IPT_PREC_F64) v = IPT_UNSUPPORTED;
  if (v == IPT_OK && opt.accel != IPT_ACCEL_NONE && opt.accel != IPT_ACCEL_ACX)
    v = IPT_UNSUPPORTED;
  const bool acx = opt.accel == IPT_ACCEL_ACX;
  if (v != IPT_OK) {
    out->status = v;
    return v;
  }
  DeviceGuard g(h->dev);
  const auto t_start = std::chrono::steady_clock::now();
  h->launches = 0;
  Timing tm;
  tm.on = opt.record_timing != 0;
  if (tm.on && ensure_events(h) != IPT_OK) {
    out->status = IPT_CUDA_ERROR;
    return IPT_CUDA_ERROR;
  }
  const bool f64 = prec == IPT_PREC_F64;
  const int ni = (int)n, ki = (int)k, kk = (int)round_up(k, 64);
  const size_t ez = f64 ? 8 : 4, nk = (size_t)n * kk;
  int nsm = 0, dev = 0;  // persistent SpMM grid: 8 CTAs of 256 threads per SM
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nblk = (nsm > 0 ? nsm : 148) * 8;
  CK(ensure(h->z[0], nk * ez));
  CK(ensure(h->z[1], nk * ez));
  if (acx) {  // f^2(z), f^3(z), the inner evaluations' d and the step lengths
    CK(ensure(h->z[2], nk * ez));
    CK(ensure(h->z[3], nk * ez));
    CK(ensure(h->acx_d, (size_t)kk * 2 * 8));
    CK(ensure(h->acx_acc, (size_t)kk * 2 * 8));
    CK(ensure(h->acx_sigma, (size_t)kk * 8));
  }
  CK(ensure(h->theta, (size_t)n * 8));
  CK(ensure(h->thh, (size_t)n * 4));
  CK(ensure(h->thl, (size_t)n * 4));
  CK(ensure(h->delta, (size_t)n * 12));  // FP64 delta_j, then its FP32 copy
  CK(ensure(h->icol, (size_t)kk * 4));
  CK(ensure(h->count, (size_t)n * 4));
  CK(ensure(h->d, (size_t)kk * 8));
  CK(ensure(h->st, sizeof(DevState)));
  CK(ensure(h->cpart, (size_t)((n + 255) / 256) * 8));  // one partial per row-pass block
  cudaStream_t s = h->s;
  DevState* st = dst(h);
  if (tm.on) cudaEventRecord(h->ev[4], s);
  CK(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  {
    DevState& init = *h->hinit;  // pinned: the copy below is truly asynchronous
    memset(&init, 0, kStateHead);
    init.stage = prec;
    init.passes = 1;
    init.accurate = 1;
    init.base = -1;
    init.z_lo = ni;
    init.z_hi = -1;
    init.nz_lo = ni;
    init.nz_hi = -1;
    init.win_lo = 0;
    init.win_hi = ni;
    CK(cudaMemcpyAsync(st, h->hinit, kStateHead, cudaMemcpyHostToDevice, s));
  }
  // Z buffers: zero everywhere but at the unit entries.  Only rows a previous
  // sparse solve of the same layout may have written need clearing.
  const bool known = h->csr_n == ni && h->csr_kk == kk && h->csr_es == (int)ez &&
                     h->csr_z[0] == h->z[0].p && h->csr_z[1] == h->z[1].p;
  const size_t row_bytes = (size_t)kk * ez;
  const size_t clr_lo = known ? (size_t)h->csr_dirty_lo : 0;
  const size_t clr_hi = known ? (size_t)h->csr_dirty_hi : (size_t)n;
  for (int b = 0; b < 2; ++b)
    if (clr_hi > clr_lo)
      CK(cudaMemsetAsync((char*)h->z[b].p + clr_lo * row_bytes, 0, (clr_hi - clr_lo) * row_bytes,
                         s));
  if (acx) {  // buffers 2 and 3 are written only inside the windows of this solve
    CK(cudaMemsetAsync(h->z[2].p, 0, nk * ez, s));
    CK(cudaMemsetAsync(h->z[3].p, 0, nk * ez, s));
    CK(cudaMemsetAsync(h->acx_acc.p, 0, (size_t)kk * 2 * 8, s));
  }
  h->csr_n = -1;  // contents unknown until this solve ends
  CK(cudaMemsetAsync(h->count.p, 0, (size_t)n * 4, s));
  launch_validate_csr(cols, ni, ki, kk, (int32_t*)h->icol.p, (int*)h->count.p, h->z[0].p,
                      f64 ? 1 : 0, st, s);
  launch_csr_rows(rowptr, colind, vals, v_dtype, theta, ni, nnz, (const int*)h->count.p,
                  (double*)h->theta.p, (float*)h->thh.p, (float*)h->thl.p, (double*)h->delta.p,
                  (double*)h->cpart.p, opt.csr_window ? 1 : 0, st, s);
  h->launches += 2;
  CK(cudaGetLastError());
  if (tm.on) cudaEventRecord(h->ev[5], s);
  ControlArgs ca;
  ca.tol = tol;
  ca.diverge_bound = opt.diverge_bound;
  ca.stage_switch = opt.stage_switch;
  ca.max_iter = max_iter;
  ca.stop = opt.stop;
  ca.mode = prec;
  ca.k = ki;
  ca.low_stage = prec;
  ca.high_stage = prec;
  // error model: the SpMM's short FP32 row sums and the FP32 map arithmetic,
  // together taken as 2^-22 of ||R0|| (FP64: 2^-51); the guard as for dense solves
  ca.e_arith = f64 ? ldexp(1.0, -51) : ldexp(1.0, -22);
  ca.guard = 1;
  ca.csr_n = ni;
  ca.csr_window = opt.csr_window ? 1 : 0;
  // IPT-ACX (Alg. 3) on the sparse path: buffer 0 holds z, buffers 1..3 f(z),
  // f^2(z), f^3(z) (row-major like the Picard iterates); an extrapolation of
  // order p evaluates F at z (tested; d in the handle's d, so Lambda is z's) and
  // at f(z) [, f^2(z)], then moves z in place over the window rows and widens
  // the window by the band.  One host synchronisation per extrapolation.
  for (int step = 0, done_evals = 0; acx && done_evals < max_iter; ++step) {
    const int order = (step % 2 == 0) ? 3 : 2;
    const int planned = std::min(order, max_iter - done_evals);
    double* dinner = (double*)h->acx_d.p;
    for (int q = 0; q < planned; ++q) {
      double* dq = q == 0 ? (double*)h->d.p : dinner + (size_t)(q - 1) * kk;
      h->launches += launch_csr_evaluate(
          rowptr, colind, vals, v_dtype, (const double*)h->delta.p, (const double*)h->theta.p,
          (const float*)h->thh.p, (const float*)h->thl.p, (const int32_t*)h->icol.p, dq, ni, ki,
          kk, h->z[q].p, h->z[q + 1].p, f64 ? 1 : 0, nblk, st, s,
          tm.on ? h->evb + 4 * q : nullptr);
      ControlArgs cq = ca;
      cq.acx = 1;
      cq.test = q == 0 ? 1 : 0;
      launch_control(st, cq, s, true);
      h->launches += 1;
    }
    if (planned == order) {
      launch_acx_combine_rm(h->z[0].p, h->z[1].p, h->z[2].p, h->z[order == 3 ? 3 : 2].p,
                            f64 ? 1 : 0, order, ni, ki, kk, opt.csr_window ? 1 : 0,
                            opt.acx_sigma, (double*)h->acx_acc.p, (double*)h->acx_sigma.p, st,
                            nblk / 2, s);
      h->launches += opt.csr_window ? 4 : 3;
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h->hst, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      v = IPT_CUDA_ERROR;
      break;
    }
    if (step == 0) {
      v = status_from_flags(h->hst->flags);
      if (v != IPT_OK) break;
      if (tm.on) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]) == cudaSuccess) tm.setup_ms = ms;
      }
    }
    if (tm.on) {
      const int ran = std::min(planned, h->hst->iter - done_evals);
      for (int q = 0; q < ran; ++q) collect_timing(h, 1, &tm, h->evb + 4 * q);
    }
    done_evals = h->hst->iter;
    if (h->hst->done) break;
  }
  // Evaluations are enqueued kCsrChunk at a time with one host sync per chunk:
  // every kernel returns at entry once the controller has stopped, and with
  // two Z buffers the iterate alternates (evaluation i reads buffer i & 1).
  for (int it0 = 0; !acx && it0 < max_iter; it0 += kCsrChunk) {
    const int nb = std::min(kCsrChunk, max_iter - it0);
    for (int q = 0; q < nb; ++q) {
      const int cur = (it0 + q) & 1;
      h->launches += launch_csr_evaluate(
          rowptr, colind, vals, v_dtype, (const double*)h->delta.p, (const double*)h->theta.p,
          (const float*)h->thh.p, (const float*)h->thl.p, (const int32_t*)h->icol.p,
          (double*)h->d.p, ni, ki, kk, h->z[cur].p, h->z[cur ^ 1].p, f64 ? 1 : 0, nblk, st, s,
          tm.on ? h->evb + 4 * q : nullptr);
      launch_control(st, ca, s, true);
      h->launches += 1;
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h->hst, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      v = IPT_CUDA_ERROR;
      break;
    }
    if (it0 == 0) {
      v = status_from_flags(h->hst->flags);
      if (v != IPT_OK) break;
      if (tm.on) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[4], h->ev[5]) == cudaSuccess) tm.setup_ms = ms;
      }
    }
    if (tm.on) {  // the evaluations of this chunk that ran before the stop
      const int ran = std::min(nb, h->hst->iter - it0);
      for (int q = 0; q < ran; ++q) {
        float a_ = 0.f, b_ = 0.f;
        if (cudaEventElapsedTime(&a_, h->evb[4 * q], h->evb[4 * q + 1]) == cudaSuccess)
          tm.prepass_ms += a_;
        if (cudaEventElapsedTime(&b_, h->evb[4 * q + 2], h->evb[4 * q + 3]) == cudaSuccess)
          tm.product_ms[0] += b_;
        tm.product_launches[0] += 1;
      }
    }
    if (h->hst->done) break;
  }
  if (v != IPT_OK) {
    out->status = v;
    return v;
  }
  // the whole state came back with the last loop synchronisation, after which
  // no kernel of the solve ran
  const DevState& hs = *h->hst;
  if (tm.on) cudaEventRecord(h->ev[6], s);
  launch_lambda((const double*)h->theta.p, (const int32_t*)h->icol.p, (const double*)h->d.p, ki,
                lambda, s);
  // rows outside the last window are zero in the returned iterate
  const int wl = hs.win_lo, wh = hs.win_hi;
  const size_t oes = z_dtype == IPT_DTYPE_F64 ? 8 : 4;
  if (wl > 0) CK(cudaMemset2DAsync(Z, (size_t)ldz * oes, 0, (size_t)wl * oes, (size_t)ki, s));
  if (wh < ni)
    CK(cudaMemset2DAsync((char*)Z + (size_t)wh * oes, (size_t)ldz * oes, 0,
                         (size_t)(ni - wh) * oes, (size_t)ki, s));
  launch_csr_out(h->z[hs.answer].p, f64 ? 1 : 0, wl, wh, ki, kk, Z, ldz,
                 z_dtype == IPT_DTYPE_F64 ? 1 : 0, s);
  h->launches += 2;
  if (tm.on) cudaEventRecord(h->ev[7], s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    out->status = IPT_CUDA_ERROR;
    return IPT_CUDA_ERROR;
  }
  if (tm.on) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[6], h->ev[7]) == cudaSuccess) tm.finalize_ms = ms;
  }
  // both Z buffers were written only inside the (growing) windows
  h->csr_n = ni;
  h->csr_kk = kk;
  h->csr_es = (int)ez;
  h->csr_z[0] = h->z[0].p;
  h->csr_z[1] = h->z[1].p;
  h->csr_dirty_lo = wl;
  h->csr_dirty_hi = wh;
  fill_result(hs, tm, h->launches, out);
  out->wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (opt.verify_fp64) {
    // ||M Z - Z Lambda||_F of the returned pair in FP64, over all rows
    CK(ensure(h->racc, 8));
    CK(cudaMemsetAsync(h->racc.p, 0, 8, s));
    launch_csr_residual64(rowptr, colind, vals, v_dtype, ni, ki, kk, h->z[hs.answer].p,
                          f64 ? 1 : 0, lambda, (double*)h->racc.p, s);
    h->launches += 1;
    double r2 = 0.0;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&r2, h->racc.p, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out->rho_fp64 = hs.r0acc > 0.0 ? sqrt(r2) / sqrt(hs.r0acc) : 0.0;
    out->kernel_launches = h->launches;
  }
  return (ipt_status)out->status;
}

ipt_status ipt_solve_batched(ipt_handle* h, int64_t count, const int64_t* n, const float* M,
                             const double* theta, double tol, int max_iter,
                             const ipt_options* opt_in, double* lambda, float* Z, int32_t* status,
                             int32_t* iters, ipt_result* out) {
  if (!out) return IPT_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->rho_fp64 = -1.0;
  ipt_options opt;
  ipt_options_default(&opt);
  if (opt_in) opt = *opt_in;
  ipt_status v = IPT_OK;
  if (!h || count < 1 || count > (1 << 30) || !n || !M || !lambda || !Z || !status || !iters ||
      !(tol >= 0.0) || max_iter < 1 ||
      (opt.stop != IPT_STOP_INCREMENT && opt.stop != IPT_STOP_RESIDUAL))
    v = IPT_INVALID_ARG;
  int64_t max_n = 0;
  for (int64_t p = 0; v == IPT_OK && p < count; ++p) {
    if (n[p] < 1 || n[p] > kBatchMaxN) v = IPT_INVALID_ARG;
    max_n = std::max(max_n, n[p]);
  }
  if (v != IPT_OK) {
    out->status = v;
    return v;
  }
  DeviceGuard g(h->dev);
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t s = h->s;
  // schedule: offsets in input order, problems largest first
  const size_t cnt = (size_t)count;
  constexpr int kTuneSample = 64;  // problems per size class in a tuning run
  const size_t meta_main = cnt * (8 + 8 + 4 + 4 + 8);
  const size_t meta_bytes = meta_main + (size_t)kBatchClasses * kTuneSample * 4 + 64;
  if (h->hmeta_cap < meta_bytes) {
    if (h->hmeta) cudaFreeHost(h->hmeta);
    h->hmeta = nullptr;
    h->hmeta_cap = 0;
    CK(cudaMallocHost(&h->hmeta, meta_bytes));
    h->hmeta_cap = meta_bytes;
  }
  int64_t* m_off = static_cast<int64_t*>(h->hmeta);
  int64_t* v_off = m_off + cnt;
  int* nsz = reinterpret_cast<int*>(v_off + cnt);
  int* order = nsz + cnt;
  int64_t* t_off = reinterpret_cast<int64_t*>(order + cnt);  // tensor-core tile sets
  int* sample = reinterpret_cast<int*>(t_off + cnt);  // kBatchClasses x kTuneSample schedules
  int64_t mo = 0, vo = 0, to = 0;
  for (size_t p = 0; p < cnt; ++p) {
    m_off[p] = mo;
    v_off[p] = vo;
    t_off[p] = to;
    nsz[p] = (int)n[p];
    order[p] = (int)p;
    mo += n[p] * n[p];
    vo += n[p];
    to += batched_tc_tile_bytes(n[p]);
  }
  std::stable_sort(order, order + cnt, [&](int a, int b) { return nsz[a] > nsz[b]; });
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // BF16 tensor-core products (split x3 or one pass) or the FP32 SIMT product
  const int tc_passes =
      opt.precision == IPT_PREC_BF16X3 ? 3 : (opt.precision == IPT_PREC_BF16 ? 1 : 0);
  // tensor cores: one CTA per SM (its shared-memory ring); FP32: the occupancy
  const int per_sm = tc_passes ? 1 : batched_ctas_per_sm();
  const int ctas = (int)std::min<int64_t>(count, (int64_t)nsm * per_sm);
  const int64_t max_n2 = max_n * max_n;
  // the tuning schedules: up to kTuneSample problems of each class not tuned yet,
  // evenly spread over the class (largest first)
  int nsample[kBatchClasses] = {};
  if (!tc_passes) {
    std::vector<int> members[kBatchClasses];
    for (size_t i = 0; i < cnt; ++i) members[batch_class_host(nsz[order[i]])].push_back(order[i]);
    for (int c = 0; c < kBatchClasses; ++c) {
      if (h->btiles[c] != 0 || members[c].empty()) continue;
      const size_t m = members[c].size(), take = std::min<size_t>(m, kTuneSample);
      for (size_t q = 0; q < take; ++q)
        sample[c * kTuneSample + q] = members[c][q * m / take];
      nsample[c] = (int)take;
    }
  }
  CK(ensure(h->bmeta, meta_bytes + 16));
  // tensor cores: the CTAs' workspaces, then the prologue's per-problem outputs
  const size_t ws_all = ((size_t)ctas * (size_t)batched_tc_workspace(max_n) + 1023) / 1024 * 1024;
  CK(ensure(h->bscratch, tc_passes ? ws_all + (size_t)batched_tc_prep_bytes(to, mo, (int)count, max_n)
                                   : (size_t)ctas * 2 * (size_t)max_n2 * 4));
  char* dm = static_cast<char*>(h->bmeta.p);
  int* queue = reinterpret_cast<int*>(dm + meta_bytes - 64);
  const int64_t* d_moff = reinterpret_cast<const int64_t*>(dm);
  const int64_t* d_voff = d_moff + cnt;
  const int* d_nsz = reinterpret_cast<const int*>(dm + cnt * 16);
  const int* d_order = reinterpret_cast<const int*>(dm + cnt * 20);
  const int64_t* d_toff = reinterpret_cast<const int64_t*>(dm + cnt * 24);
  const int* d_sample = reinterpret_cast<const int*>(dm + meta_main);
  bool tune = false;
  for (int c = 0; c < kBatchClasses; ++c) tune |= nsample[c] > 0;
  if (tune) CK(cudaMemcpyAsync(dm, h->hmeta, meta_bytes - 64, cudaMemcpyHostToDevice, s));
  Timing tm;
  tm.on = opt.record_timing != 0;
  if (ensure_events(h) != IPT_OK) {
    out->status = IPT_CUDA_ERROR;
    return IPT_CUDA_ERROR;
  }
  // autotuner: for every size class met for the first time, time each output
  // tile on a sample of the class's problems and keep the faster (the tuning
  // runs write outputs that the full run below overwrites)
  for (int c = 0; c < kBatchClasses; ++c) {
    if (!nsample[c]) continue;
    float best_ms = 0.f;
    int best = 64;
    for (int tile : {64, 32}) {
      int tiles[kBatchClasses] = {64, 64, 64};
      tiles[c] = tile;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first run warms caches and the clock
        CK(cudaMemsetAsync(queue, 0, sizeof(int), s));
        CK(cudaEventRecord(h->ev[0], s));
        CK(launch_batched(M, theta, d_moff, d_voff, d_nsz, d_sample + c * kTuneSample,
                          nsample[c], max_n2, tol, max_iter, opt.stop, opt.diverge_bound,
                          lambda, Z, status, iters, static_cast<float*>(h->bscratch.p), queue,
                          tiles, std::min(ctas, nsample[c]), s));
        CK(cudaEventRecord(h->ev[1], s));
        CK(cudaEventSynchronize(h->ev[1]));
        CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
      }
      if (tile == 64 || ms < best_ms) {
        best_ms = ms;
        best = tile;
      }
    }
    h->btiles[c] = best;
  }
  int tiles[kBatchClasses];
  for (int c = 0; c < kBatchClasses; ++c) tiles[c] = h->btiles[c] ? h->btiles[c] : 64;
  // the solve itself: schedule copy, queue reset and kernel as one CUDA graph,
  // captured once per set of arguments and replayed while they repeat
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](uint64_t x) { key = (key ^ x) * 1099511628211ull; };
  for (size_t p = 0; p < cnt; ++p) mix((uint64_t)nsz[p]);
  const void* ptrs[] = {M, theta, lambda, Z, status, iters, h->bscratch.p, h->bmeta.p, h->hmeta};
  for (const void* q : ptrs) mix(reinterpret_cast<uintptr_t>(q));
  uint64_t tb;
  memcpy(&tb, &tol, 8);
  mix(tb);
  memcpy(&tb, &opt.diverge_bound, 8);
  mix(tb);
  mix((uint64_t)max_iter);
  mix((uint64_t)opt.stop);
  mix((uint64_t)cnt);
  mix((uint64_t)ctas);
  for (int c = 0; c < kBatchClasses; ++c) mix((uint64_t)tiles[c]);
  mix((uint64_t)tc_passes);
  if (!h->bexec || h->bkey != key) {
    if (h->bexec) cudaGraphExecDestroy(h->bexec);
    if (h->bgraph) cudaGraphDestroy(h->bgraph);
    h->bexec = nullptr;
    h->bgraph = nullptr;
    if (!h->gs) CK(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking));
    cudaStream_t cs = h->gs;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(dm, h->hmeta, meta_main, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(queue, 0, sizeof(int), cs);
    if (tc_passes)
      launch_batched_tc(M, theta, d_moff, d_voff, d_toff, d_nsz, d_order, (int)count, max_n, to,
                        mo, tol, max_iter, opt.stop, opt.diverge_bound, lambda, Z, status,
                        iters, h->bscratch.p, static_cast<char*>(h->bscratch.p) + ws_all, queue,
                        ctas, tc_passes, cs);
    else
      launch_batched(M, theta, d_moff, d_voff, d_nsz, d_order, (int)count, max_n2, tol,
                     max_iter, opt.stop, opt.diverge_bound, lambda, Z, status, iters,
                     static_cast<float*>(h->bscratch.p), queue, tiles, ctas, cs);
    CK(cudaStreamEndCapture(cs, &h->bgraph));
    CK(cudaGraphInstantiate(&h->bexec, h->bgraph, 0));
    h->bkey = key;
  }
  if (tm.on) cudaEventRecord(h->ev[2], s);
  CK(cudaGraphLaunch(h->bexec, s));
  if (tm.on) cudaEventRecord(h->ev[3], s);
  // per-problem outcomes for the aggregate result
  const size_t stat_bytes = cnt * 2 * sizeof(int);
  if (h->hstat_cap < stat_bytes) {
    if (h->hstat) cudaFreeHost(h->hstat);
    h->hstat = nullptr;
    h->hstat_cap = 0;
    CK(cudaMallocHost((void**)&h->hstat, stat_bytes));
    h->hstat_cap = stat_bytes;
  }
  CK(cudaMemcpyAsync(h->hstat, status, cnt * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->hstat + cnt, iters, cnt * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int agg = IPT_OK, most = 0;
  for (size_t p = 0; p < cnt; ++p) {
    if (agg == IPT_OK && h->hstat[p] != IPT_OK) agg = h->hstat[p];
    most = std::max(most, h->hstat[cnt + p]);
  }
  out->status = agg;
  out->iterations = most;
  out->kernel_launches = tc_passes ? 2 : 1;  // tensor cores: the prologue and the solve
  out->product_launches[0] = 1;
  if (tm.on) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]) == cudaSuccess) out->product_ms[0] = ms;
  }
  out->wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return (ipt_status)agg;
}

ipt_status ipt_check_bounded_wait(int arrive, double limit_s, void* stream, int32_t* succeeded,
                                  double* waited_s) {
  if (!succeeded || !(limit_s > 0.0) || limit_s > 10.0) return IPT_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(long long)) != cudaSuccess) return IPT_CUDA_ERROR;
  long long hv[2] = {0, 0};
  const bool ok =
      launch_wait_check(arrive ? 1 : 0, (uint64_t)(limit_s * 1e9), d, s) == cudaSuccess &&
      cudaMemcpyAsync(hv, d, sizeof(hv), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
      cudaStreamSynchronize(s) == cudaSuccess;
  cudaFree(d);
  if (!ok) return IPT_CUDA_ERROR;
  *succeeded = (int32_t)hv[0];
  if (waited_s) *waited_s = (double)hv[1] * 1e-9;
  return IPT_OK;
}

ipt_status ipt_check_map_division(int64_t count, const float* gap, const float* u,
                                  float* quotient, void* stream) {
  if (count < 0 || (count > 0 && (!gap || !u || !quotient))) return IPT_INVALID_ARG;
  return launch_recip_check(count, gap, u, quotient, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_check_conversions(int64_t count, const double* x, float* hi, float* lo,
                                 float* f, double* back, int32_t* ok, void* stream) {
  if (count < 0 || (count > 0 && (!x || !hi || !lo || !f || !back || !ok)))
    return IPT_INVALID_ARG;
  return launch_conv_check(count, x, hi, lo, f, back, ok, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_set_batched_tiles(ipt_handle* h, const int32_t* tiles) {
  if (!h || !tiles) return IPT_INVALID_ARG;
  for (int c = 0; c < kBatchClasses; ++c)
    if (tiles[c] != 0 && tiles[c] != 32 && tiles[c] != 64) return IPT_INVALID_ARG;
  for (int c = 0; c < kBatchClasses; ++c) h->btiles[c] = tiles[c];
  return IPT_OK;
}

ipt_status ipt_get_batched_tiles(const ipt_handle* h, int32_t* tiles) {
  if (!h || !tiles) return IPT_INVALID_ARG;
  for (int c = 0; c < kBatchClasses; ++c) tiles[c] = h->btiles[c];
  return IPT_OK;
}

ipt_status ipt_damping_forward(int64_t B, const void* params, const float* x, float* alpha,
                               void* stream) {
  if (B < 0 || B > (int64_t)1 << 30 || (B > 0 && (!params || !x || !alpha)))
    return IPT_INVALID_ARG;
  return launch_mlp_forward(params, x, (int)B, alpha, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_damping_grad(int64_t B, const void* params, const float* x, const float* target,
                            float* grad, double* loss, void* stream) {
  if (B < 0 || B > (int64_t)1 << 30 || !grad || !loss ||
      (B > 0 && (!params || !x || !target)))
    return IPT_INVALID_ARG;
  return launch_mlp_grad(params, x, target, (int)B, grad, loss,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_damping_adam(float* master, void* params, float* grad, float* m, float* v,
                            float lr, float beta1, float beta2, float eps, int step,
                            void* stream) {
  if (!master || !params || !grad || !m || !v || step < 1) return IPT_INVALID_ARG;
  return launch_mlp_adam(master, params, grad, m, v, lr, beta1, beta2, eps, step,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_mixing_forward(int64_t B, const void* params, const float* x, float* out,
                              void* stream) {
  if (B < 0 || B > (int64_t)1 << 30 || (B > 0 && (!params || !x || !out)))
    return IPT_INVALID_ARG;
  return launch_mix_forward(params, x, (int)B, out, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_mixing_grad(int64_t B, const void* params, const float* x, const float* target,
                           float* grad, double* loss, void* stream) {
  if (B < 0 || B > (int64_t)1 << 30 || !grad || !loss ||
      (B > 0 && (!params || !x || !target)))
    return IPT_INVALID_ARG;
  return launch_mix_grad(params, x, target, (int)B, grad, loss,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

ipt_status ipt_mixing_adam(float* master, void* params, float* grad, float* m, float* v,
                           float lr, float beta1, float beta2, float eps, int step,
                           void* stream) {
  if (!master || !params || !grad || !m || !v || step < 1) return IPT_INVALID_ARG;
  return launch_mix_adam(master, params, grad, m, v, lr, beta1, beta2, eps, step,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? IPT_OK
             : IPT_CUDA_ERROR;
}

}  // extern "C"
