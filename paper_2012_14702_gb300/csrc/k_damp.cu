// Learned damping on the device: after an evaluation F(Z) (written to its own
// buffer) the next iterate Z + alpha_c (F(Z) - Z) replaces F there, one alpha per column, alpha_c from the damping
// model (k_mlp.cu) fed the column's history of increment norms and
// Rayleigh-quotient changes.  The first three steps (no history yet) and
// every step after the fallback has tripped are plain Picard steps
// (alpha = 1): the fallback trips when a step's residual exceeds ten times
// the smallest residual seen, or an alpha is not finite.
//
// Features of column c (oldest .. newest increments i2, i1, i0 and
// eigenvalues l2, l1, l0; eps = 1e-30):
//   log10(i0 + eps), log10((i0 + eps)/(i1 + eps)), log10((i1 + eps)/(i2 + eps)),
//   clip((l0 - l1)/(l1 - l2), -4, 4) (0 if l1 = l2),
//   log10(|l1 - l2|/(|l1| + eps) + eps), log10(|l0 - l1|/(|l0| + eps) + eps).
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int RPT = 4;  // rows per thread

// Per column: ||F_c - Z_c||^2 and ||Z_c||^2 (block partials into acc[2c],
// acc[2c+1]), accumulated in the iterate's precision (the history features
// need a few digits; FP64 per entry would run on the slow FP64 pipe).
template <typename T>
__global__ void __launch_bounds__(256)
    k_damp_colnorms(const T* __restrict__ z, const T* __restrict__ f, int n, int64_t ld,
                    double* __restrict__ acc, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  const int64_t col = (int64_t)c * ld;
  T a = T(0), b = T(0);
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = (blockIdx.y * RPT + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      const T zv = z[col + j], dv = f[col + j] - zv;
      a = fma(dv, dv, a);
      b = fma(zv, zv, b);
    }
  }
  __shared__ T ra[8], rb[8];
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T s = T(0), t = T(0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s += ra[w];
      t += rb[w];
    }
    atomicAdd(&acc[2 * c], (double)s);
    atomicAdd(&acc[2 * c + 1], (double)t);
  }
}

// Per column: the new history entry, the features when three are known, and
// the flag whether the model's alpha is used.  Clears acc.  One thread (c = 0)
// also runs the fallback test on the evaluation's residual.
__global__ void k_damp_prepare(double* __restrict__ acc, const double* __restrict__ theta,
                               const int32_t* __restrict__ icol, const double* __restrict__ d,
                               int k, float* __restrict__ hinc, double* __restrict__ hlam,
                               float* __restrict__ X, DampState* ds, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int steps = ds->steps;  // histories recorded before this one
  if (c == 0) {
    const double rho = st->rho;
    if (steps == 0 || rho < ds->best_rho) ds->best_rho = rho;
    if (steps >= 3 && rho > 10.0 * ds->best_rho) ds->fallback = 1;
  }
  if (c >= k) return;
  const double a = acc[2 * c], b = acc[2 * c + 1];
  acc[2 * c] = acc[2 * c + 1] = 0.0;
  const float inc = b > 0.0 ? (float)sqrt(a / b) : 0.f;
  // eigenvalue history in FP64: its differences are far below FP32's
  // resolution of the eigenvalues themselves
  const double lam = theta[icol[c]] + d[c];
  // history rows t-2, t-1, t (k entries each)
  const float i2 = hinc[k + c], i1 = hinc[2 * k + c];
  const double l2 = hlam[k + c], l1 = hlam[2 * k + c];
  hinc[c] = i2;
  hinc[k + c] = i1;
  hinc[2 * k + c] = inc;
  hlam[c] = l2;
  hlam[k + c] = l1;
  hlam[2 * k + c] = lam;
  if (steps + 1 < 3) return;
  const float e = 1e-30f;
  const double num = lam - l1, den = l1 - l2;
  const float q = den != 0.0 ? (float)fmin(fmax(num / den, -4.0), 4.0) : 0.f;
  float* x = X + (int64_t)c * kMlpInputs;
  x[0] = log10f(inc + e);
  x[1] = log10f((inc + e) / (i1 + e));
  x[2] = log10f((i1 + e) / (i2 + e));
  x[3] = q;
  x[4] = log10f((float)(fabs(den) / (fabs(l1) + 1e-30)) + e);
  x[5] = log10f((float)(fabs(num) / (fabs(lam) + 1e-30)) + e);
}

__global__ void k_damp_count(DampState* ds, const DevState* st) {
  if (st->done) return;
  ds->steps += 1;
}

// F's buffer <- Z + alpha_c (F - Z): the next iterate (alpha_c = 1 before the
// model applies or after the fallback leaves F as it is).  Grid (column, row block).
template <typename T>
__global__ void __launch_bounds__(256)
    k_damp_update(const T* __restrict__ z, T* __restrict__ f, int n, int64_t ld,
                  const float* __restrict__ alpha, const DampState* ds, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  if (ds->steps < 3 || ds->fallback) return;
  float a = alpha[c];
  if (!isfinite(a)) a = 1.f;
  const int64_t col = (int64_t)c * ld;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = (blockIdx.y * RPT + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      const T zv = z[col + j];
      f[col + j] = zv + (T)a * (f[col + j] - zv);
    }
  }
}

}  // namespace

cudaError_t launch_damp_step(const void* z, void* f, int f64, int n, int k, int64_t ld,
                             const double* theta, const int32_t* icol, const double* d,
                             const void* model, double* acc, float* hinc, double* hlam,
                             float* X, float* alpha, DampState* ds, DevState* st,
                             cudaStream_t s) {
  const dim3 g((unsigned)k, (unsigned)((n + 256 * RPT - 1) / (256 * RPT)));
  if (f64)
    k_damp_colnorms<double><<<g, 256, 0, s>>>((const double*)z, (const double*)f, n, ld, acc, st);
  else
    k_damp_colnorms<float><<<g, 256, 0, s>>>((const float*)z, (const float*)f, n, ld, acc, st);
  k_damp_prepare<<<(k + 255) / 256, 256, 0, s>>>(acc, theta, icol, d, k, hinc, hlam, X, ds,
                                                 st);
  k_damp_count<<<1, 1, 0, s>>>(ds, st);
  cudaError_t e = launch_mlp_forward(model, X, k, alpha, s);
  if (e != cudaSuccess) return e;
  if (f64)
    k_damp_update<double><<<g, 256, 0, s>>>((const double*)z, (double*)f, n, ld, alpha, ds, st);
  else
    k_damp_update<float><<<g, 256, 0, s>>>((const float*)z, (float*)f, n, ld, alpha, ds, st);
  return cudaGetLastError();
}

}  // namespace ipt
