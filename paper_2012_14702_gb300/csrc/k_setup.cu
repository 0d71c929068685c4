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
// Non-finite theta is flagged here; equal theta_j == theta_{cols[c]} is
// detected where the product epilogues form the gap (gap == 0 off the
// unit entry), at no extra pass over the n x k pairs.
__global__ void k_theta(const void* M, int64_t ldm, int m_dtype, const double* theta_in, int n,
                        int npad, double* theta, float* th_hi, float* th_lo, DevState* st) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npad) return;
  double t = 0.0;
  if (j < n) t = theta_in ? theta_in[j] : load_m(M, (int64_t)j * ldm + j, m_dtype);
  if (j < n && !isfinite(t)) atomicOr(&st->flags, FLAG_THETA_NONFINITE);
  theta[j] = t;
  float h = (float)t;
  th_hi[j] = h;
  th_lo[j] = (float)(t - (double)h);
}

// icol[c] = cols[c] (or c), range check, occurrence count per index.
__global__ void k_cols(const int32_t* cols, int n, int k, int kpad, int32_t* icol, int* count,
                       DevState* st, int col_range, void* zunit, int kk, int zf64) {
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
  if (col_range) {  // the support of Z0 = E: rows [z_lo, z_hi] (sparse solves)
    atomicMin(&st->z_lo, i);
    atomicMax(&st->z_hi, i);
  }
  if (zunit) {  // Z0 = E in the sparse path's row-major n x kk iterate
    if (zf64) static_cast<double*>(zunit)[(int64_t)i * kk + c] = 1.0;
    else static_cast<float*>(zunit)[(int64_t)i * kk + c] = 1.f;
  }
}

// Duplicate requested columns (after k_cols has counted occurrences).
__global__ void k_cols_dup(const int32_t* icol, const int* count, int k, DevState* st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int i = icol[c];
  if (i >= 0 && count[i] > 1) atomicOr(&st->flags, FLAG_COL_DUP);
}

// Delta = M - diag(theta) (Alg. 1/2 step 1).  Off-diagonal entries are M's
// own values, copied without arithmetic; the n diagonal ones are formed in
// FP64 before rounding, M_ii - theta_i (theta_i ~ 1e3 would otherwise swamp
// Delta_ii ~ 1e-3 in any 16- or 32-bit format).  Stored as FP64/FP32
// row-major and (optionally) FP32 column-major, transposed through shared
// memory.  Also sums the squared off-diagonal entries of the requested
// columns (the residual normaliser ||R0||^2).  Block 32x8, tile 32x32.
template <typename TM, typename TD>
__global__ void k_form_delta(const TM* __restrict__ M, int64_t ldm, const double* theta, int n,
                             int npad, const int* count, TD* __restrict__ Drow,
                             float* __restrict__ DT, float* __restrict__ r0part) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = c0 + tx;
  const bool req = j < n && count[j] > 0;
  float r0sum = 0.f;
  for (int q = 0; q < 4; ++q) {
    const int i = r0 + ty + 8 * q;
    TD v = TD(0);
    if (i < n && j < n) {
      if (i == j) {
        v = (TD)((double)M[(int64_t)i * ldm + j] - theta[i]);
      } else {
        v = (TD)M[(int64_t)i * ldm + j];
        if (req) r0sum = fmaf((float)v, (float)v, r0sum);
      }
    }
    Drow[(int64_t)i * npad + j] = v;
    tile[ty + 8 * q][tx] = (float)v;
  }
  if (DT) {
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int jj = c0 + ty + 8 * q, i = r0 + tx;
      DT[(int64_t)jj * npad + i] = tile[tx][ty + 8 * q];
    }
  }
  // block partial of ||R0||^2 (one slot per block; summed by k_sum_partials)
  __shared__ float red[8];
  const float w = warp_sum(r0sum);
  if (tx == 0) red[ty] = w;
  __syncthreads();
  if (tx == 0 && ty == 0) {
    float t = 0.f;
    for (int q = 0; q < 8; ++q) t += red[q];
    r0part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// The same for FP32 M with 16-byte aligned rows: tile 64 x 64, block 16 x 16.
// Each thread moves 4 consecutive columns of 4 rows with 16-byte loads and
// stores (a row segment is 256 contiguous bytes); the transposed FP32 copy
// goes through a 65-float padded shared tile and leaves as 256-byte column
// segments (one float2 per lane).  The diagonal entries are copied as M_ii
// by the streaming loop and then replaced, in the tiles on the diagonal only,
// by M_ii - theta_i formed in FP64 (the FP64 pipe is far slower than the
// FP32 one here: no per-entry FP64 work, not even a predicated one).
__device__ __noinline__ float diag_delta(float m, double theta) {
  return (float)((double)m - theta);
}

__global__ void __launch_bounds__(256)
    k_form_delta4(const float* __restrict__ M, int64_t ldm, const double* theta, int n,
                  int npad, const int* count, float* __restrict__ Drow, float* __restrict__ DT,
                  float* __restrict__ r0part) {
  __shared__ float tile[64][65];
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = c0 + 4 * tx;
  bool req[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) req[u] = (j + u < n) && count[j + u] > 0;
  float r0sum = 0.f;
  float4 m4[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // all loads first
    const int i = r0 + ty + 16 * q;
    m4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
      if (j + 3 < n) {
        m4[q] = *reinterpret_cast<const float4*>(M + (int64_t)i * ldm + j);
      } else {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        for (int u = 0; u < 4; ++u)
          if (j + u < n) t[u] = M[(int64_t)i * ldm + j + u];
        m4[q] = make_float4(t[0], t[1], t[2], t[3]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = r0 + ty + 16 * q;
    const float v[4] = {m4[q].x, m4[q].y, m4[q].z, m4[q].w};
    if (i < n) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j + u != i && req[u]) r0sum = fmaf(v[u], v[u], r0sum);
    }
    *reinterpret_cast<float4*>(Drow + (int64_t)i * npad + j) = m4[q];
#pragma unroll
    for (int u = 0; u < 4; ++u) tile[ty + 16 * q][4 * tx + u] = v[u];
  }
  const int tid = ty * 16 + tx, lane = tid & 31, w = tid >> 5;
  if (blockIdx.x == blockIdx.y) {  // a tile on the diagonal: Delta_ii = M_ii - theta_i
    __syncthreads();
    const int i = r0 + tid;
    if (tid < 64 && i < n) {
      const float dv = diag_delta(tile[tid][tid], theta[i]);
      tile[tid][tid] = dv;
      Drow[(int64_t)i * npad + i] = dv;
    }
  }
  if (DT) {
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {  // 8 warps x 8 columns, rows 2 lane, 2 lane + 1
      const int col = w * 8 + cc;
      *reinterpret_cast<float2*>(DT + (int64_t)(c0 + col) * npad + r0 + 2 * lane) =
          make_float2(tile[2 * lane][col], tile[2 * lane + 1][col]);
    }
  }
  __shared__ float red[8];
  const float ws = warp_sum(r0sum);
  if (lane == 0) red[w] = ws;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int q = 0; q < 8; ++q) t += red[q];
    r0part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// One block: st->r0acc = sum of the per-block FP32 partials (as FP32 pairs,
// in a fixed order).
__global__ void __launch_bounds__(1024)
    k_sum_partials(const float* __restrict__ part, int64_t count, DevState* st) {
  __shared__ F2 sh[32];
  F2 t{0.f, 0.f};
#pragma unroll 4
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) t = f2_add(t, F2{part[i], 0.f});
  t = block_sum(t, sh);
  if (threadIdx.x == 0) st->r0acc = f2_value(t);
}

// Tensor-core A operand: row j of Delta scaled by the power of two r_j that
// brings its largest entry into [2^13, 2^14), split into 16-bit hi + lo.
// One CTA per row (all npad rows; padding rows are zero); the row stays in
// registers between the max and the split (VPT float4 per thread).
template <int VPT>
__global__ void __launch_bounds__(1024)
    k_split_delta(const float* __restrict__ Drow, int npad, int bf16,
                  uint16_t* __restrict__ Dh, uint16_t* __restrict__ Dl,
                  float* __restrict__ rinv) {
  const int row = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n4 = npad / 4;
  const float4* a = reinterpret_cast<const float4*>(Drow + (int64_t)row * npad);
  float4 x[VPT];
  float mx = 0.f;
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const int m = tid + q * blockDim.x;
    x[q] = m < n4 ? __ldg(a + m) : make_float4(0.f, 0.f, 0.f, 0.f);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x[q].x), fabsf(x[q].y)), fmaxf(fabsf(x[q].z), fabsf(x[q].w))));
  }
  __shared__ float rm[32];
  mx = warp_max(mx);
  if (lane == 0) rm[wid] = mx;
  __syncthreads();
  float rmax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rmax = fmaxf(rmax, rm[w]);
  const float sc = pow2_scale(rmax);
  uint2* h2 = reinterpret_cast<uint2*>(Dh + (int64_t)row * npad);
  uint2* l2 = reinterpret_cast<uint2*>(Dl + (int64_t)row * npad);
#pragma unroll
  for (int q = 0; q < VPT; ++q) {
    const int m = tid + q * blockDim.x;
    if (m < n4) {
      uint16_t h[4], l[4];
      split16(x[q].x * sc, bf16, h[0], l[0]);
      split16(x[q].y * sc, bf16, h[1], l[1]);
      split16(x[q].z * sc, bf16, h[2], l[2]);
      split16(x[q].w * sc, bf16, h[3], l[3]);
      h2[m] = make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
      l2[m] = make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
    }
  }
  if (tid == 0) rinv[row] = 1.f / sc;
}

// Rows longer than 4 * 8 * 1024 entries: one warp per row, two passes.
__global__ void k_split_delta_wide(const float* __restrict__ Drow, int npad, int bf16,
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

template <typename TZ>
__device__ __forceinline__ void init_z_entry(const void* z0, int64_t ldz0, int z0_dtype,
                                             const int32_t* icol, int n, int k, int npad, int c,
                                             int j, TZ* Z, DevState* st) {
  const int i = icol[c];
  TZ z = TZ(0);
  if (c < k && j < n && i >= 0) {
    if (z0) {
      double piv = load_m(z0, (int64_t)c * ldz0 + i, z0_dtype);
      if (piv == 0.0 || !isfinite(piv)) {
        if (j == i) atomicOr(&st->flags, FLAG_ZERO_PIVOT);
        piv = 1.0;
      }
      z = (j == i) ? TZ(1) : (TZ)(load_m(z0, (int64_t)c * ldz0 + j, z0_dtype) / piv);
    } else {
      z = (j == i) ? TZ(1) : TZ(0);
    }
  }
  Z[(int64_t)c * npad + j] = z;
}

// Z = unit columns E (or the rescaled warm start), padding zero.
// Grid (ceil(npad/1024), kpad): blockIdx.y is the column, 4 rows per thread.
template <typename TZ>
__global__ void k_init_z(const void* z0, int64_t ldz0, int z0_dtype, const int32_t* icol, int n,
                         int k, int npad, TZ* Z, DevState* st) {
  const int c = blockIdx.y;
  for (int q = 0; q < 4; ++q) {
    const int j = (blockIdx.x * 4 + q) * blockDim.x + threadIdx.x;
    if (j < npad) init_z_entry(z0, ldz0, z0_dtype, icol, n, k, npad, c, j, Z, st);
  }
}

// Lambda_c = theta_{i_c} + d_c (Alg. 2: Lambda = D(M Z), Z_{i_c, c} = 1).
__global__ void k_lambda(const double* theta, const int32_t* icol, const double* d, int k,
                         double* lambda) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < k) lambda[c] = theta[icol[c]] + d[c];
}

// Grid (ceil(n/1024), k): blockIdx.y is the column, 4 rows per thread.
template <typename TI, typename TO>
__global__ void k_copy_z(const TI* __restrict__ Z, int64_t ld, int n, TO* __restrict__ out,
                         int64_t ldo) {
  const int c = blockIdx.y;
  const TI* src = Z + (int64_t)c * ld;
  TO* dst = out + (int64_t)c * ldo;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = (blockIdx.x * 4 + q) * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = (TO)src[j];
  }
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
                  int npad, double* theta, float* th_hi, float* th_lo, DevState* st,
                  cudaStream_t s) {
  k_theta<<<blocks(npad, 256), 256, 0, s>>>(M, ldm, m_dtype, theta_in, n, npad, theta, th_hi,
                                            th_lo, st);
}

void launch_validate(const int32_t* cols, int n, int k, int kpad, const double* theta,
                     int32_t* icol, int* count, DevState* st, cudaStream_t s) {
  (void)theta;
  k_cols<<<blocks(kpad, 256), 256, 0, s>>>(cols, n, k, kpad, icol, count, st, 0, nullptr, 0, 0);
  k_cols_dup<<<blocks(k, 256), 256, 0, s>>>(icol, count, k, st);
}

void launch_validate_csr(const int32_t* cols, int n, int k, int kk, int32_t* icol, int* count,
                         void* Z, int zf64, DevState* st, cudaStream_t s) {
  k_cols<<<blocks(kk, 256), 256, 0, s>>>(cols, n, k, kk, icol, count, st, 1, Z, kk, zf64);
}

void launch_form_delta(const void* M, int64_t ldm, int m_dtype, const double* theta, int n,
                       int npad, const int* count, void* Drow, int drow_f64, float* DT,
                       double* r0part_d, DevState* st, cudaStream_t s) {
  float* r0part = reinterpret_cast<float*>(r0part_d);  // per-block FP32 partials
  dim3 b(32, 8);
  if (m_dtype == IPT_DTYPE_F32 && !drow_f64 && ldm % 4 == 0 &&
      (reinterpret_cast<uintptr_t>(M) & 15) == 0) {
    dim3 g4(npad / 64, npad / 64), b4(16, 16);
    k_form_delta4<<<g4, b4, 0, s>>>((const float*)M, ldm, theta, n, npad, count, (float*)Drow,
                                    DT, r0part);
    k_sum_partials<<<1, 1024, 0, s>>>(r0part, (int64_t)g4.x * g4.y, st);
    return;
  }
  dim3 g(npad / 32, npad / 32);
  if (m_dtype == IPT_DTYPE_F64 && drow_f64)
    k_form_delta<double, double><<<g, b, 0, s>>>((const double*)M, ldm, theta, n, npad, count,
                                                 (double*)Drow, DT, r0part);
  else if (m_dtype == IPT_DTYPE_F64)
    k_form_delta<double, float><<<g, b, 0, s>>>((const double*)M, ldm, theta, n, npad, count,
                                                (float*)Drow, DT, r0part);
  else if (drow_f64)
    k_form_delta<float, double><<<g, b, 0, s>>>((const float*)M, ldm, theta, n, npad, count,
                                                (double*)Drow, DT, r0part);
  else
    k_form_delta<float, float><<<g, b, 0, s>>>((const float*)M, ldm, theta, n, npad, count,
                                               (float*)Drow, DT, r0part);
  k_sum_partials<<<1, 1024, 0, s>>>(r0part, (int64_t)g.x * g.y, st);
}

void launch_split_delta(const float* Drow, int npad, int bf16, uint16_t* Dh, uint16_t* Dl,
                        float* rinv, cudaStream_t s) {
  constexpr int VPT = 8;
  const int n4 = npad / 4;
  if (n4 <= VPT * 1024) {
    int threads = ((n4 + VPT - 1) / VPT + 31) / 32 * 32;
    k_split_delta<VPT><<<npad, threads, 0, s>>>(Drow, npad, bf16, Dh, Dl, rinv);
  } else {
    k_split_delta_wide<<<(unsigned)((npad + 7) / 8), 256, 0, s>>>(Drow, npad, bf16, Dh, Dl, rinv);
  }
}

void launch_init_z(const void* z0, int64_t ldz0, int z0_dtype, const int32_t* icol, int n,
                   int k, int npad, int kpad, void* Z, int z_f64, DevState* st, cudaStream_t s) {
  dim3 g(blocks(npad, 1024), kpad);
  if (z_f64)
    k_init_z<double><<<g, 256, 0, s>>>(z0, ldz0, z0_dtype, icol, n, k, npad, (double*)Z, st);
  else
    k_init_z<float><<<g, 256, 0, s>>>(z0, ldz0, z0_dtype, icol, n, k, npad, (float*)Z, st);
}

void launch_lambda(const double* theta, const int32_t* icol, const double* d, int k,
                   double* lambda, cudaStream_t s) {
  k_lambda<<<blocks(k, 256), 256, 0, s>>>(theta, icol, d, k, lambda);
}

void launch_copy_z(const void* Z, int z_f64, int64_t ld, int n, int k, void* out, int64_t ldo,
                   int out_f64, cudaStream_t s) {
  dim3 g(blocks(n, 1024), k);
  if (z_f64 && out_f64)
    k_copy_z<double, double><<<g, 256, 0, s>>>((const double*)Z, ld, n, (double*)out, ldo);
  else if (z_f64)
    k_copy_z<double, float><<<g, 256, 0, s>>>((const double*)Z, ld, n, (float*)out, ldo);
  else if (out_f64)
    k_copy_z<float, double><<<g, 256, 0, s>>>((const float*)Z, ld, n, (double*)out, ldo);
  else
    k_copy_z<float, float><<<g, 256, 0, s>>>((const float*)Z, ld, n, (float*)out, ldo);
}

void launch_convert_m64(const void* M, int64_t ldm, int m_dtype, int n, int npad, double* M64,
                        cudaStream_t s) {
  k_convert_m64<<<blocks((int64_t)npad * npad, 256), 256, 0, s>>>(M, ldm, m_dtype, n, npad, M64);
}

}  // namespace ipt
