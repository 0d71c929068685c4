// Setup kernels: the partition M = D + Delta (Alg. 1/2 step 1, Section 3),
// argument validation on the device, the starting point Z = I (or a warm
// start) and result copies.  All run once per solve; O(n^2) or O(nk) work.
#include "ipt_internal.cuh"

#include <math.h>

namespace ipt {

namespace {

__device__ __forceinline__ double load_m(const void* M, int64_t idx, int m_dtype) {
  return m_dtype == IPT_DTYPE_F64 ? static_cast<const double*>(M)[idx]
                                  : static_cast<double>(static_cast<const float*>(M)[idx]);
}

// theta (given, or diag(M)) and its two-float split; padding rows get 0.
__global__ void k_theta(const void* M, int64_t ldm, int m_dtype, const double* theta_in, int n,
                        int npad, double* theta, float* th_hi, float* th_lo) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npad) return;
  double t = 0.0;
  if (j < n) t = theta_in ? theta_in[j] : load_m(M, (int64_t)j * ldm + j, m_dtype);
  theta[j] = t;
  float h = (float)t;
  th_hi[j] = h;
  th_lo[j] = (float)(t - (double)h);
}

// icol[c] = cols[c] (or c), range check, occurrence count per index.
__global__ void k_cols(const int32_t* cols, int n, int k, int kpad, int32_t* icol, int* count,
                       DevState* st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kpad) return;
  if (c >= k) {
    icol[c] = -1;
    return;
  }
  int i = cols ? cols[c] : c;
  if (i < 0 || i >= n) {
    atomicOr(&st->flags, FLAG_COL_RANGE);
    icol[c] = -1;
    return;
  }
  icol[c] = i;
  atomicAdd(&count[i], 1);
}

// Duplicate columns, non-finite theta, theta_j == theta_{cols[c]} (j != cols[c]).
// Grid: (k, ceil(n / (blockDim*4))).
__global__ void k_theta_check(const double* theta, const int32_t* icol, const int* count, int n,
                              DevState* st) {
  int c = blockIdx.x;
  int i = icol[c];
  if (i < 0) return;
  double ti = theta[i];
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    if (count[i] > 1) atomicOr(&st->flags, FLAG_COL_DUP);
    if (!isfinite(ti)) atomicOr(&st->flags, FLAG_THETA_NONFINITE);
  }
  int base = blockIdx.y * blockDim.x * 4;
  bool bad = false;
  for (int q = 0; q < 4; ++q) {
    int j = base + q * blockDim.x + threadIdx.x;
    if (j < n && j != i) {
      double tj = theta[j];
      bad |= (tj == ti) || !isfinite(tj);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    atomicOr(&st->flags, FLAG_THETA_DEGENERATE);
}

// Delta = M - diag(theta), formed in FP64 before any rounding, then stored
// as FP64/FP32 row-major and (optionally) FP32 column-major, transposed
// through shared memory.  Also sums the squared off-diagonal entries of the
// requested columns (the residual normaliser ||R0||^2).  Block 32x8, tile 32x32.
__global__ void k_form_delta(const void* M, int64_t ldm, int m_dtype, const double* theta, int n,
                             int npad, const int* count, void* Drow, int drow_f64, float* DT,
                             DevState* st) {
  __shared__ float tile[32][33];
  int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  int tx = threadIdx.x, ty = threadIdx.y;
  double r0sum = 0.0;
  for (int q = 0; q < 4; ++q) {
    int i = r0 + ty + 8 * q, j = c0 + tx;
    double v = 0.0;
    if (i < n && j < n) {
      v = load_m(M, (int64_t)i * ldm + j, m_dtype);
      if (i == j) v -= theta[i];
      else if (count[j] > 0) r0sum += v * v;
    }
    int64_t o = (int64_t)i * npad + j;
    if (drow_f64) static_cast<double*>(Drow)[o] = v;
    else static_cast<float*>(Drow)[o] = (float)v;
    tile[ty + 8 * q][tx] = (float)v;
  }
  if (DT) {
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      int j = c0 + ty + 8 * q, i = r0 + tx;
      DT[(int64_t)j * npad + i] = tile[tx][ty + 8 * q];
    }
  }
  r0sum = warp_sum(r0sum);
  if (tx == 0 && r0sum != 0.0) atomicAdd(&st->r0acc, r0sum);
}

// Tensor-core A operand: row j of Delta scaled by the power of two r_j that
// brings its largest entry into [2^13, 2^14), split into 16-bit hi + lo.
// One warp per row (all npad rows; padding rows are zero).
__global__ void k_split_delta(const float* __restrict__ Drow, int npad, int bf16,
                              uint16_t* __restrict__ Dh, uint16_t* __restrict__ Dl,
                              float* __restrict__ rinv) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= npad) return;
  const float4* a = reinterpret_cast<const float4*>(Drow + (int64_t)row * npad);
  float mx = 0.f;
  for (int m = lane; m < npad / 4; m += 32) {
    const float4 x = a[m];
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
  }
  mx = warp_max(mx);
  const float sc = pow2_scale(mx);
  uint2* h2 = reinterpret_cast<uint2*>(Dh + (int64_t)row * npad);
  uint2* l2 = reinterpret_cast<uint2*>(Dl + (int64_t)row * npad);
  for (int m = lane; m < npad / 4; m += 32) {
    const float4 x = a[m];
    uint16_t h[4], l[4];
    split16(x.x * sc, bf16, h[0], l[0]);
    split16(x.y * sc, bf16, h[1], l[1]);
    split16(x.z * sc, bf16, h[2], l[2]);
    split16(x.w * sc, bf16, h[3], l[3]);
    h2[m] = make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
    l2[m] = make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
  }
  if (lane == 0) rinv[row] = 1.f / sc;
}

// Z = unit columns E (or the rescaled warm start), padding zero.
template <typename TZ>
__global__ void k_init_z(const void* z0, int64_t ldz0, int z0_dtype, const int32_t* icol, int n,
                         int k, int npad, int kpad, TZ* Z, DevState* st) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)kpad * npad;
  if (idx >= total) return;
  int c = (int)(idx / npad), j = (int)(idx % npad);
  int i = icol[c];
  double z = 0.0;
  if (c < k && j < n && i >= 0) {
    if (z0) {
      double piv = load_m(z0, (int64_t)c * ldz0 + i, z0_dtype);
      if (piv == 0.0 || !isfinite(piv)) {
        if (j == i) atomicOr(&st->flags, FLAG_ZERO_PIVOT);
        piv = 1.0;
      }
      z = (j == i) ? 1.0 : load_m(z0, (int64_t)c * ldz0 + j, z0_dtype) / piv;
    } else {
      z = (j == i) ? 1.0 : 0.0;
    }
  }
  Z[idx] = (TZ)z;
}

// Lambda_c = theta_{i_c} + d_c (Alg. 2: Lambda = D(M Z), Z_{i_c, c} = 1).
__global__ void k_lambda(const double* theta, const int32_t* icol, const double* d, int k,
                         double* lambda) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < k) lambda[c] = theta[icol[c]] + d[c];
}

template <typename TI, typename TO>
__global__ void k_copy_z(const TI* Z, int64_t ld, int n, int k, TO* out, int64_t ldo) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * k) return;
  int c = (int)(idx / n), j = (int)(idx % n);
  out[(int64_t)c * ldo + j] = (TO)Z[(int64_t)c * ld + j];
}

__global__ void k_convert_m64(const void* M, int64_t ldm, int m_dtype, int n, int npad,
                              double* M64) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)npad * npad) return;
  int i = (int)(idx / npad), j = (int)(idx % npad);
  M64[idx] = (i < n && j < n) ? load_m(M, (int64_t)i * ldm + j, m_dtype) : 0.0;
}

inline unsigned blocks(int64_t total, int bs) { return (unsigned)((total + bs - 1) / bs); }

}  // namespace

void launch_theta(const void* M, int64_t ldm, int m_dtype, const double* theta_in, int n,
                  int npad, double* theta, float* th_hi, float* th_lo, cudaStream_t s) {
  k_theta<<<blocks(npad, 256), 256, 0, s>>>(M, ldm, m_dtype, theta_in, n, npad, theta, th_hi,
                                            th_lo);
}

void launch_validate(const int32_t* cols, int n, int k, int kpad, const double* theta,
                     int32_t* icol, int* count, DevState* st, cudaStream_t s) {
  k_cols<<<blocks(kpad, 256), 256, 0, s>>>(cols, n, k, kpad, icol, count, st);
  dim3 g(k, (unsigned)((n + 1023) / 1024));
  k_theta_check<<<g, 256, 0, s>>>(theta, icol, count, n, st);
}

void launch_form_delta(const void* M, int64_t ldm, int m_dtype, const double* theta, int n,
                       int npad, const int* count, void* Drow, int drow_f64, float* DT,
                       DevState* st, cudaStream_t s) {
  dim3 g(npad / 32, npad / 32), b(32, 8);
  k_form_delta<<<g, b, 0, s>>>(M, ldm, m_dtype, theta, n, npad, count, Drow, drow_f64, DT, st);
}

void launch_split_delta(const float* Drow, int npad, int bf16, uint16_t* Dh, uint16_t* Dl,
                        float* rinv, cudaStream_t s) {
  k_split_delta<<<(unsigned)((npad + 7) / 8), 256, 0, s>>>(Drow, npad, bf16, Dh, Dl, rinv);
}

void launch_init_z(const void* z0, int64_t ldz0, int z0_dtype, const int32_t* icol, int n,
                   int k, int npad, int kpad, void* Z, int z_f64, DevState* st, cudaStream_t s) {
  int64_t total = (int64_t)kpad * npad;
  if (z_f64)
    k_init_z<double><<<blocks(total, 256), 256, 0, s>>>(z0, ldz0, z0_dtype, icol, n, k, npad,
                                                        kpad, (double*)Z, st);
  else
    k_init_z<float><<<blocks(total, 256), 256, 0, s>>>(z0, ldz0, z0_dtype, icol, n, k, npad,
                                                       kpad, (float*)Z, st);
}

void launch_lambda(const double* theta, const int32_t* icol, const double* d, int k,
                   double* lambda, cudaStream_t s) {
  k_lambda<<<blocks(k, 256), 256, 0, s>>>(theta, icol, d, k, lambda);
}

void launch_copy_z(const void* Z, int z_f64, int64_t ld, int n, int k, void* out, int64_t ldo,
                   int out_f64, cudaStream_t s) {
  unsigned g = blocks((int64_t)n * k, 256);
  if (z_f64 && out_f64)
    k_copy_z<double, double><<<g, 256, 0, s>>>((const double*)Z, ld, n, k, (double*)out, ldo);
  else if (z_f64)
    k_copy_z<double, float><<<g, 256, 0, s>>>((const double*)Z, ld, n, k, (float*)out, ldo);
  else if (out_f64)
    k_copy_z<float, double><<<g, 256, 0, s>>>((const float*)Z, ld, n, k, (double*)out, ldo);
  else
    k_copy_z<float, float><<<g, 256, 0, s>>>((const float*)Z, ld, n, k, (float*)out, ldo);
}

void launch_convert_m64(const void* M, int64_t ldm, int m_dtype, int n, int npad, double* M64,
                        cudaStream_t s) {
  k_convert_m64<<<blocks((int64_t)npad * npad, 256), 256, 0, s>>>(M, ldm, m_dtype, n, npad, M64);
}

}  // namespace ipt
