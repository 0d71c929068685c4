// Learned damping and mixing on the device (accel = IPT_ACCEL_MIXING).  After
// the evaluation g_t = F(z_t) of Eq. (dyn) each column c moves to
//   z_{t+1} = z_t + alpha f_t - gamma ((z_t - z_{t-1}) + alpha (f_t - f_{t-1})),
// f = g - z, with (alpha_c, gamma_c) from the mixing model (k_mlp.cu) fed the
// damping model's six history features and the least-squares Anderson weight
// gamma_ls = <f_t - f_{t-1}, f_t> / ||f_t - f_{t-1}||^2 (clipped to +-4).  The
// first three steps (no history yet) and every step after the fallback has
// tripped (a residual above ten times the smallest seen, or a non-finite
// output) are Picard steps (alpha = 1, gamma = 0).  Both map values are 1 at
// the unit entry, so every iterate keeps it.
//
// FP64 iterates: FP64 arithmetic; FP32 iterates: FP32 per element, FP64
// accumulators per column.  Every kernel returns at entry once the controller
// has stopped the solve.
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int RPT = 4;  // rows per thread

// Per column: ||f||^2, ||z||^2 and, with a previous pair, <df, f>, ||df||^2
// (df = f_t - f_{t-1}); block partials into acc[4c .. 4c+3].  Grid (column, row block).
template <typename T>
__global__ void __launch_bounds__(256)
    k_mix_stats(const T* __restrict__ z, const T* __restrict__ g, const T* __restrict__ zp,
                const T* __restrict__ gp, int n, int64_t ld, double* __restrict__ acc,
                const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  const int64_t col = (int64_t)c * ld;
  T s[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = (blockIdx.y * RPT + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      const T zv = z[col + j], f = g[col + j] - zv;
      s[0] = fma(f, f, s[0]);
      s[1] = fma(zv, zv, s[1]);
      if (zp) {
        const T df = f - (gp[col + j] - zp[col + j]);
        s[2] = fma(df, f, s[2]);
        s[3] = fma(df, df, s[3]);
      }
    }
  }
  __shared__ T red[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T v = warp_sum(s[i]);
    if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    T a = T(0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[threadIdx.x][w];
    if (a != T(0)) atomicAdd(&acc[4 * c + threadIdx.x], (double)a);
  }
}

// Per column: the history entry, the seven features once three are known, and
// the clearing of acc; thread 0 runs the fallback test on the evaluation's
// residual (stored by the controller in st->rho).
__global__ void k_mix_prepare(double* __restrict__ acc, const double* __restrict__ theta,
                              const int32_t* __restrict__ icol, const double* __restrict__ d,
                              int k, float* __restrict__ hinc, double* __restrict__ hlam,
                              float* __restrict__ X, DampState* ms, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int steps = ms->steps;  // histories recorded before this one
  if (c == 0) {
    const double rho = st->rho;
    if (steps == 0 || rho < ms->best_rho) ms->best_rho = rho;
    if (steps >= 3 && rho > 10.0 * ms->best_rho) ms->fallback = 1;
  }
  if (c >= k) return;
  const double ff = acc[4 * c], zz = acc[4 * c + 1], num = acc[4 * c + 2],
               den = acc[4 * c + 3];
  acc[4 * c] = acc[4 * c + 1] = acc[4 * c + 2] = acc[4 * c + 3] = 0.0;
  const float inc = zz > 0.0 ? (float)sqrt(ff / zz) : 0.f;
  const double lam = theta[icol[c]] + d[c];  // FP64: its changes are below FP32's resolution
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
  const double dn = lam - l1, dd = l1 - l2;
  const float q = dd != 0.0 ? (float)fmin(fmax(dn / dd, -4.0), 4.0) : 0.f;
  const double gls = den > 0.0 ? num / den : 0.0;
  float* x = X + (int64_t)c * kMixInputs;
  x[0] = log10f(inc + e);
  x[1] = log10f((inc + e) / (i1 + e));
  x[2] = log10f((i1 + e) / (i2 + e));
  x[3] = q;
  x[4] = log10f((float)(fabs(dd) / (fabs(l1) + 1e-30)) + e);
  x[5] = log10f((float)(fabs(dn) / (fabs(lam) + 1e-30)) + e);
  x[6] = (float)fmin(fmax(gls, -4.0), 4.0);
}

__global__ void k_mix_count(DampState* ms, const DevState* st) {
  if (st->done) return;
  ms->steps += 1;
}

// out <- z + alpha f - gamma ((z - zp) + alpha (f - fp)) with (alpha, gamma) =
// (1, 0) before the model applies or after the fallback.  `out` is zp's buffer:
// every element is read before it is written, by the same thread.
template <typename T>
__global__ void __launch_bounds__(256)
    k_mix_update(T* __restrict__ out, const T* __restrict__ z, const T* __restrict__ g,
                 const T* __restrict__ zp, const T* __restrict__ gp, int n, int64_t ld,
                 const float* __restrict__ ag, const DampState* ms, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  float a = 1.f, gm = 0.f;
  if (ms->steps >= 3 && !ms->fallback) {
    a = ag[2 * c];
    gm = ag[2 * c + 1];
    if (!isfinite(a) || !isfinite(gm)) {
      a = 1.f;
      gm = 0.f;
    }
  }
  const T A = (T)a, Gm = (T)gm;
  const int64_t col = (int64_t)c * ld;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = (blockIdx.y * RPT + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      const T zv = z[col + j], f = g[col + j] - zv;
      const T zq = zp[col + j], fq = gp[col + j] - zq;
      out[col + j] = zv + A * f - Gm * ((zv - zq) + A * (f - fq));
    }
  }
}

}  // namespace

cudaError_t launch_mix_step(const void* z, const void* g, const void* zp, const void* gp,
                            void* out, int f64, int n, int k, int64_t ld, const double* theta,
                            const int32_t* icol, const double* d, const void* model,
                            double* acc, float* hinc, double* hlam, float* X, float* ag,
                            DampState* ms, DevState* st, cudaStream_t s) {
  const dim3 grid((unsigned)k, (unsigned)((n + 256 * RPT - 1) / (256 * RPT)));
  if (f64)
    k_mix_stats<double><<<grid, 256, 0, s>>>((const double*)z, (const double*)g,
                                             (const double*)zp, (const double*)gp, n, ld, acc,
                                             st);
  else
    k_mix_stats<float><<<grid, 256, 0, s>>>((const float*)z, (const float*)g, (const float*)zp,
                                            (const float*)gp, n, ld, acc, st);
  k_mix_prepare<<<(k + 255) / 256, 256, 0, s>>>(acc, theta, icol, d, k, hinc, hlam, X, ms, st);
  k_mix_count<<<1, 1, 0, s>>>(ms, st);  // the model applies once three histories are known
  cudaError_t e = launch_mix_forward(model, X, k, ag, s);
  if (e != cudaSuccess) return e;
  if (zp) {  // with a previous pair; the first step is a Picard step (z_1 = g_0 in place)
    if (f64)
      k_mix_update<double><<<grid, 256, 0, s>>>((double*)out, (const double*)z,
                                                (const double*)g, (const double*)zp,
                                                (const double*)gp, n, ld, ag, ms, st);
    else
      k_mix_update<float><<<grid, 256, 0, s>>>((float*)out, (const float*)z, (const float*)g,
                                               (const float*)zp, (const float*)gp, n, ld, ag, ms,
                                               st);
  }
  return cudaGetLastError();
}

}  // namespace ipt
