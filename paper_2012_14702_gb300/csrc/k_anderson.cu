// Anderson mixing of depth one in place of the Picard update (accel =
// IPT_ACCEL_ANDERSON).  After the evaluation g_t = F(z_t) of Eq. (dyn), each
// column c takes
//   gamma_c = <f_t - f_{t-1}, f_t> / ||f_t - f_{t-1}||^2,   f = g - z
//   z_{t+1} = g_t - gamma_c (g_t - g_{t-1})
// (gamma_c = 0 when the difference vanishes, at the first step, and for every
// step after a residual rose above ten times the smallest one seen).  Both
// map values are 1 at the unit entry, so z_{t+1} keeps it.
//
// FP64 iterates: FP64 arithmetic.  FP32 iterates: FP32 per element (the FP64
// pipe runs at a small fraction of the FP32 rate here), FP64 accumulators per
// column.  Every kernel returns at entry once the controller has stopped.
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int RPT = 4;  // rows per thread

// Per column: <df, f> and ||df||^2 (df = f_t - f_{t-1}) over rows; block
// partials into acc[2c], acc[2c + 1].  Grid (column, row block).
template <typename T>
__global__ void __launch_bounds__(256)
    k_and_dots(const T* __restrict__ z, const T* __restrict__ g, const T* __restrict__ zp,
               const T* __restrict__ gp, int n, int64_t ld, double* __restrict__ acc,
               const AndState* as, const DevState* st) {
  if (st->done || as->steps == 0) return;
  const int c = blockIdx.x;
  const int64_t col = (int64_t)c * ld;
  T num = T(0), den = T(0);
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = (blockIdx.y * RPT + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      const T f = g[col + j] - z[col + j], fq = gp[col + j] - zp[col + j];
      const T df = f - fq;
      num = fma(df, f, num);
      den = fma(df, df, den);
    }
  }
  __shared__ T rn[8], rd[8];
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    rn[threadIdx.x >> 5] = num;
    rd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T a = T(0), b = T(0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += rn[w];
      b += rd[w];
    }
    atomicAdd(&acc[2 * c], (double)a);
    atomicAdd(&acc[2 * c + 1], (double)b);
  }
}

// Per column: gamma_c (clearing the accumulators); thread 0 keeps the
// smallest residual and trips the fallback (the controller has stored this
// evaluation's residual in st->rho).
__global__ void k_and_gamma(double* __restrict__ acc, int k, double* __restrict__ gamma,
                            AndState* as, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int steps = as->steps;  // evaluations before this one
  const double rho = st->rho;
  const double best = (steps == 0 || rho < as->best_rho) ? rho : as->best_rho;
  const bool fallback = as->fallback || (steps > 0 && rho > 10.0 * best);
  if (c < k) {
    const double num = acc[2 * c], den = acc[2 * c + 1];
    acc[2 * c] = acc[2 * c + 1] = 0.0;
    gamma[c] = (steps == 0 || fallback || !(den > 0.0)) ? 0.0 : num / den;
  }
  if (c == 0) {
    as->best_rho = best;
    as->fallback = fallback ? 1 : 0;
  }
}

__global__ void k_and_count(AndState* as, const DevState* st) {
  if (st->done) return;
  as->steps += 1;
}

// out <- g - gamma_c (g - g_prev).  `out` may be the buffer of z_{t-1}
// (each element is read by the dots kernel before and written once here).
template <typename T>
__global__ void __launch_bounds__(256)
    k_and_update(T* __restrict__ out, const T* __restrict__ g, const T* __restrict__ gp, int n,
                 int64_t ld, const double* __restrict__ gamma, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  const int64_t col = (int64_t)c * ld;
  const T gm = (T)gamma[c];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int j = (blockIdx.y * RPT + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      const T a = g[col + j];
      out[col + j] = a - gm * (a - gp[col + j]);
    }
  }
}

}  // namespace

cudaError_t launch_anderson_step(const void* z, const void* g, const void* zp, const void* gp,
                                 void* out, int f64, int n, int k, int64_t ld, double* acc,
                                 double* gamma, AndState* as, DevState* st, int first,
                                 cudaStream_t s) {
  const dim3 grid((unsigned)k, (unsigned)((n + 256 * RPT - 1) / (256 * RPT)));
  if (first) {  // a Picard step: z_1 = g_0 stays in g's buffer; only the state advances
    k_and_gamma<<<(k + 255) / 256, 256, 0, s>>>(acc, k, gamma, as, st);
    k_and_count<<<1, 1, 0, s>>>(as, st);
    return cudaGetLastError();
  }
  if (f64)
    k_and_dots<double><<<grid, 256, 0, s>>>((const double*)z, (const double*)g,
                                            (const double*)zp, (const double*)gp, n, ld, acc, as,
                                            st);
  else
    k_and_dots<float><<<grid, 256, 0, s>>>((const float*)z, (const float*)g, (const float*)zp,
                                           (const float*)gp, n, ld, acc, as, st);
  k_and_gamma<<<(k + 255) / 256, 256, 0, s>>>(acc, k, gamma, as, st);
  if (f64)
    k_and_update<double><<<grid, 256, 0, s>>>((double*)out, (const double*)g, (const double*)gp,
                                              n, ld, gamma, st);
  else
    k_and_update<float><<<grid, 256, 0, s>>>((float*)out, (const float*)g, (const float*)gp, n,
                                             ld, gamma, st);
  k_and_count<<<1, 1, 0, s>>>(as, st);
  return cudaGetLastError();
}

}  // namespace ipt
