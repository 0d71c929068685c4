// Alternating Cyclic Extrapolation (Alg. 3, Section 5) on the device: after
// an extrapolation's evaluations z -> f(z) -> f^2(z) [-> f^3(z)] the iterate
// moves to
//   p = 2:  z + 2 s D1 + s^2 D2
//   p = 3:  z + 3 s D1 + 3 s^2 D2 + s^3 D3
// with the differences D1 = f - z, D2 = f^2 - 2 f + z,
// D3 = f^3 - 3 f^2 + 3 f - z and the step s = |<Dp, D(p-1)>| / ||Dp||^2 of
// each column (or one s for the whole block); a column with Dp = 0 takes
// s = 1, which makes the update the plain iterate f^p(z).
//
// Iterates are column-major (element (j, c) at c * ld + j).  FP64 iterates:
// differences, inner products and the update in FP64.  FP32 iterates: in
// FP32 (the FP64 pipe runs at a small fraction of the FP32 rate here), with
// the higher differences formed from first differences of consecutive
// iterates (f - z, f^2 - f, f^3 - f^2), which are exact whenever the two
// entries lie within a factor of two of each other (Sterbenz) and otherwise
// carry one rounding relative to themselves; per-block sums go to FP64
// accumulators.  Every kernel returns at entry once the controller has
// stopped the solve.
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int ROWS_PER_THREAD = 4;

__device__ __forceinline__ void differences(const double* z, const double* f1, const double* f2,
                                            const double* f3, int64_t o, int p, double& d1,
                                            double& d2, double& d3) {
  const double x = z[o], a = f1[o], b = f2[o];
  d1 = a - x;
  d2 = b - 2.0 * a + x;
  d3 = p == 3 ? (f3[o] - 3.0 * b + 3.0 * a - x) : 0.0;
}

__device__ __forceinline__ void differences(const float* z, const float* f1, const float* f2,
                                            const float* f3, int64_t o, int p, float& d1,
                                            float& d2, float& d3) {
  const float x = z[o], a = f1[o], b = f2[o];
  const float e1 = a - x, e2 = b - a;
  d1 = e1;
  d2 = e2 - e1;
  d3 = p == 3 ? ((f3[o] - b) - e2) - d2 : 0.f;
}

// Per column: <Dp, D(p-1)> and ||Dp||^2 over rows, block partials added
// into the FP64 acc[2c], acc[2c + 1].  Grid (column, row block).
template <typename T>
__global__ void __launch_bounds__(256)
    k_acx_dots(const T* __restrict__ z, const T* __restrict__ f1, const T* __restrict__ f2,
               const T* __restrict__ f3, int p, int n, int64_t ld, double* __restrict__ acc,
               const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  const int64_t col = (int64_t)c * ld;
  T num = T(0), den = T(0);
#pragma unroll
  for (int q = 0; q < ROWS_PER_THREAD; ++q) {
    const int j = (blockIdx.y * ROWS_PER_THREAD + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      T d1, d2, d3;
      differences(z, f1, f2, f3, col + j, p, d1, d2, d3);
      const T dp = p == 3 ? d3 : d2, dq = p == 3 ? d2 : d1;
      num = fma(dp, dq, num);
      den = fma(dp, dp, den);
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

// One block: the step of every column (or the global step) into sigma[c];
// clears acc for the next extrapolation.
__global__ void __launch_bounds__(1024)
    k_acx_sigma(double* __restrict__ acc, int k, int global, double* __restrict__ sigma,
                const DevState* st) {
  if (st->done) return;
  __shared__ double rn[1024], rd[1024];
  if (global) {
    double a = 0.0, b = 0.0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      a += acc[2 * c];
      b += acc[2 * c + 1];
    }
    rn[threadIdx.x] = a;
    rd[threadIdx.x] = b;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) {
        rn[threadIdx.x] += rn[threadIdx.x + h];
        rd[threadIdx.x] += rd[threadIdx.x + h];
      }
      __syncthreads();
    }
    const double s = rd[0] > 0.0 ? fabs(rn[0]) / rd[0] : 1.0;
    for (int c = threadIdx.x; c < k; c += blockDim.x) sigma[c] = s;
  } else {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      const double a = acc[2 * c], b = acc[2 * c + 1];
      sigma[c] = b > 0.0 ? fabs(a) / b : 1.0;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) acc[2 * c] = acc[2 * c + 1] = 0.0;
}

// z <- the order-p extrapolation, in place.  Grid (column, row block).
template <typename T>
__global__ void __launch_bounds__(256)
    k_acx_update(T* __restrict__ z, const T* __restrict__ f1, const T* __restrict__ f2,
                 const T* __restrict__ f3, int p, int n, int64_t ld,
                 const double* __restrict__ sigma, const DevState* st) {
  if (st->done) return;
  const int c = blockIdx.x;
  const int64_t col = (int64_t)c * ld;
  const T s = (T)sigma[c];
#pragma unroll
  for (int q = 0; q < ROWS_PER_THREAD; ++q) {
    const int j = (blockIdx.y * ROWS_PER_THREAD + q) * blockDim.x + threadIdx.x;
    if (j < n) {
      T d1, d2, d3;
      differences(z, f1, f2, f3, col + j, p, d1, d2, d3);
      const T x = z[col + j];
      const T y = p == 3 ? x + T(3) * s * d1 + T(3) * s * s * d2 + s * s * s * d3
                         : x + T(2) * s * d1 + s * s * d2;
      z[col + j] = y;
    }
  }
}

// Row-major iterates of the sparse path (element (j, c) at j * kk + c): only
// the rows of the state's window [win_lo, win_hi) are visited, every other row
// being zero in all four buffers.  A persistent grid strides over the rows;
// a thread owns one column of a 64-wide chunk and every fourth row.
template <typename T>
__global__ void __launch_bounds__(256)
    k_acx_dots_rm(const T* __restrict__ z, const T* __restrict__ f1, const T* __restrict__ f2,
                  const T* __restrict__ f3, int p, int k, int kk, double* __restrict__ acc,
                  const DevState* st) {
  if (st->done) return;
  const int64_t lo = st->win_lo, hi = st->win_hi;
  const int cl = threadIdx.x & 63, rq = threadIdx.x >> 6;
  __shared__ T rn[4][64], rd[4][64];
  for (int c0 = 0; c0 < kk; c0 += 64) {
    const int c = c0 + cl;
    T num = T(0), den = T(0);
    if (c < k) {
      for (int64_t j = lo + (int64_t)blockIdx.x * 4 + rq; j < hi; j += (int64_t)gridDim.x * 4) {
        T d1, d2, d3;
        differences(z, f1, f2, f3, j * kk + c, p, d1, d2, d3);
        const T dp = p == 3 ? d3 : d2, dq = p == 3 ? d2 : d1;
        num = fma(dp, dq, num);
        den = fma(dp, dp, den);
      }
    }
    rn[rq][cl] = num;
    rd[rq][cl] = den;
    __syncthreads();
    if (rq == 0 && c < k) {
      const T a = (rn[0][cl] + rn[1][cl]) + (rn[2][cl] + rn[3][cl]);
      const T b = (rd[0][cl] + rd[1][cl]) + (rd[2][cl] + rd[3][cl]);
      if (a != T(0)) atomicAdd(&acc[2 * c], (double)a);
      if (b != T(0)) atomicAdd(&acc[2 * c + 1], (double)b);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_acx_update_rm(T* __restrict__ z, const T* __restrict__ f1, const T* __restrict__ f2,
                    const T* __restrict__ f3, int p, int k, int kk,
                    const double* __restrict__ sigma, const DevState* st) {
  if (st->done) return;
  const int64_t lo = st->win_lo, hi = st->win_hi;
  const int cl = threadIdx.x & 63, rq = threadIdx.x >> 6;
  for (int c0 = 0; c0 < kk; c0 += 64) {
    const int c = c0 + cl;
    if (c >= k) continue;
    const T s = (T)sigma[c];
    for (int64_t j = lo + (int64_t)blockIdx.x * 4 + rq; j < hi; j += (int64_t)gridDim.x * 4) {
      T d1, d2, d3;
      const int64_t o = j * kk + c;
      differences(z, f1, f2, f3, o, p, d1, d2, d3);
      const T x = z[o];
      z[o] = p == 3 ? x + T(3) * s * d1 + T(3) * s * s * d2 + s * s * s * d3
                    : x + T(2) * s * d1 + s * s * d2;
    }
  }
}

// After an extrapolation of the sparse path: the new iterate is nonzero only in
// rows already evaluated, so the next product must cover them widened by the
// band (the window only grows).
__global__ void k_acx_widen(DevState* st, int n) {
  if (st->done) return;
  st->win_lo = max(0, st->win_lo - st->band);
  st->win_hi = (int)min((int64_t)n, (int64_t)st->win_hi + st->band);
}

}  // namespace

void launch_acx_combine(void* z, const void* f1, const void* f2, const void* f3, int f64, int p,
                        int n, int k, int64_t ld, int global, double* acc, double* sigma,
                        DevState* st, cudaStream_t s) {
  const dim3 g((unsigned)k, (unsigned)((n + 256 * ROWS_PER_THREAD - 1) / (256 * ROWS_PER_THREAD)));
  if (f64) {
    k_acx_dots<double><<<g, 256, 0, s>>>((const double*)z, (const double*)f1, (const double*)f2,
                                         (const double*)f3, p, n, ld, acc, st);
    k_acx_sigma<<<1, 1024, 0, s>>>(acc, k, global, sigma, st);
    k_acx_update<double><<<g, 256, 0, s>>>((double*)z, (const double*)f1, (const double*)f2,
                                           (const double*)f3, p, n, ld, sigma, st);
  } else {
    k_acx_dots<float><<<g, 256, 0, s>>>((const float*)z, (const float*)f1, (const float*)f2,
                                        (const float*)f3, p, n, ld, acc, st);
    k_acx_sigma<<<1, 1024, 0, s>>>(acc, k, global, sigma, st);
    k_acx_update<float><<<g, 256, 0, s>>>((float*)z, (const float*)f1, (const float*)f2,
                                          (const float*)f3, p, n, ld, sigma, st);
  }
}

void launch_acx_combine_rm(void* z, const void* f1, const void* f2, const void* f3, int f64,
                           int p, int n, int k, int kk, int window, int global, double* acc,
                           double* sigma, DevState* st, int blocks, cudaStream_t s) {
  if (f64) {
    k_acx_dots_rm<double><<<blocks, 256, 0, s>>>((const double*)z, (const double*)f1,
                                                 (const double*)f2, (const double*)f3, p, k, kk,
                                                 acc, st);
    k_acx_sigma<<<1, 1024, 0, s>>>(acc, k, global, sigma, st);
    k_acx_update_rm<double><<<blocks, 256, 0, s>>>((double*)z, (const double*)f1,
                                                   (const double*)f2, (const double*)f3, p, k,
                                                   kk, sigma, st);
  } else {
    k_acx_dots_rm<float><<<blocks, 256, 0, s>>>((const float*)z, (const float*)f1,
                                                (const float*)f2, (const float*)f3, p, k, kk,
                                                acc, st);
    k_acx_sigma<<<1, 1024, 0, s>>>(acc, k, global, sigma, st);
    k_acx_update_rm<float><<<blocks, 256, 0, s>>>((float*)z, (const float*)f1, (const float*)f2,
                                                  (const float*)f3, p, k, kk, sigma, st);
  }
  if (window) k_acx_widen<<<1, 1, 0, s>>>(st, n);
}

}  // namespace ipt
