// Sparse IPT evaluation: P = Delta Z for M given in CSR (all stored entries of
// M, diagonal included), with the map of Eq. (dyn) fused into the same warp.
//
// Layout.  Internally Z is row-major n x kk (kk = k rounded up to 64), so the
// gather Z[m, :] of one column index m is a single coalesced 64-wide read
// (256 B in FP32).  One warp owns one row j of Delta at a time; lane l owns
// the columns c = 64*chunk + 2l, 2l+1.  The diagonal of Delta,
// delta_j = M_jj - theta_j (0 when theta = diag(M)), is applied separately, so
// the CSR loop skips stored diagonal entries.
//
// Kernels: setup (theta, delta_j, residual normaliser, Z = E), the diagonal
// pre-pass d_c = (Delta Z)_{cols[c], c} (one warp per column: a sparse row
// dot product), the SpMM + map, and the transpose of the result to the
// column-major output of the C ABI.
#include "ipt_internal.cuh"

#include <math.h>

namespace ipt {

namespace {

template <typename T>
__device__ __forceinline__ T ldval(const void* v, int64_t i, int dt) {
  return dt == IPT_DTYPE_F64 ? (T) static_cast<const double*>(v)[i]
                             : (T) static_cast<const float*>(v)[i];
}

// theta_j (given or the stored M_jj, 0 if the row stores none), its FP32
// split, delta_j = M_jj - theta_j; non-finite theta is flagged.  One warp per row.
__global__ void k_csr_theta(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            const void* __restrict__ vals, int v_dtype,
                            const double* __restrict__ theta_in, int n, double* __restrict__ theta,
                            float* __restrict__ th_hi, float* __restrict__ th_lo,
                            double* __restrict__ delta, DevState* st) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= n) return;
  double mjj = 0.0;
  for (int e = rowptr[j] + lane; e < rowptr[j + 1]; e += 32)
    if (colind[e] == j) mjj += ldval<double>(vals, e, v_dtype);
  mjj = warp_sum(mjj);
  if (lane == 0) {
    const double t = theta_in ? theta_in[j] : mjj;
    if (!isfinite(t)) atomicOr(&st->flags, FLAG_THETA_NONFINITE);
    theta[j] = t;
    const float h = (float)t;
    th_hi[j] = h;
    th_lo[j] = (float)(t - (double)h);
    delta[j] = mjj - t;
  }
}

// ||M Z0 - Z0 Lambda0||^2: squared off-diagonal entries of the requested
// columns of M (count[col] > 0), one per-block partial.  Grid-stride over nnz.
__global__ void k_csr_r0(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                         const void* __restrict__ vals, int v_dtype, int n,
                         const int* __restrict__ count, double* __restrict__ part) {
  double s = 0.0;
  for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n;
       j += gridDim.x * (blockDim.x >> 5)) {
    for (int e = rowptr[j] + (threadIdx.x & 31); e < rowptr[j + 1]; e += 32) {
      const int m = colind[e];
      if (m != j && count[m] > 0) {
        const double v = ldval<double>(vals, e, v_dtype);
        s += v * v;
      }
    }
  }
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_csr_sum_r0(const double* __restrict__ part, int count, DevState* st) {
  __shared__ double red[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) t += part[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) st->r0acc = red[0];
}

// Z = E in the row-major layout (Z[j*kk + c] = 1 at j = cols[c]); padding zero.
template <typename T>
__global__ void k_csr_init_z(const int32_t* __restrict__ icol, int n, int kk, T* __restrict__ Z) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * kk) return;
  const int j = (int)(idx / kk), c = (int)(idx - (int64_t)j * kk);
  Z[idx] = icol[c] == j ? T(1) : T(0);
}

// d_c = sum_m Delta_{i_c, m} Z_{m, c} = delta_{i_c} Z_{i_c, c} + sum over the
// off-diagonal stored entries of row i_c.  One warp per column.
template <typename T>
__global__ void k_csr_prepass(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                              const void* __restrict__ vals, int v_dtype,
                              const double* __restrict__ delta, const int32_t* __restrict__ icol,
                              int kk, const T* __restrict__ Z, double* __restrict__ d,
                              const DevState* st) {
  if (st->done) return;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= kk) return;
  const int i = icol[c];
  if (i < 0) {
    if (lane == 0) d[c] = 0.0;
    return;
  }
  double s = 0.0;
  for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
    const int m = colind[e];
    if (m != i) s += ldval<double>(vals, e, v_dtype) * (double)Z[(int64_t)m * kk + c];
  }
  s = warp_sum(s);
  if (lane == 0) d[c] = s + delta[i] * (double)Z[(int64_t)i * kk + c];
}

template <typename T>
struct Two;
template <>
struct Two<float> {
  using V = float2;
};
template <>
struct Two<double> {
  using V = double2;
};

// SpMM + map.  Persistent: a grid of `blocks` CTAs of 8 warps walks the rows;
// each warp accumulates its row's 64-column chunk in registers (2 per lane),
// then applies the map and writes F.  Norm partials: one atomic per warp.
template <typename T>
__global__ void __launch_bounds__(256)
    k_csr_spmm_map(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                   const void* __restrict__ vals, int v_dtype, const double* __restrict__ delta,
                   const double* __restrict__ theta, const float* __restrict__ th_hi,
                   const float* __restrict__ th_lo, const int32_t* __restrict__ icol,
                   const double* __restrict__ d, int n, int k, int kk, const T* __restrict__ Zin,
                   T* __restrict__ Fout, DevState* st) {
  if (st->done) return;
  using V2 = typename Two<T>::V;
  const int lane = threadIdx.x & 31;
  const int warp0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  T s_inc = T(0), s_z = T(0), s_r = T(0);
  for (int ch = 0; ch < kk; ch += 64) {
    const int c0 = ch + 2 * lane, c1 = c0 + 1;
    const int ic0 = icol[c0], ic1 = icol[c1];
    const T d0 = (T)d[c0], d1 = (T)d[c1];
    double tc0 = 0.0, tc1 = 0.0;
    float hc0 = 0.f, lc0 = 0.f, hc1 = 0.f, lc1 = 0.f;
    if (ic0 >= 0) {
      tc0 = theta[ic0];
      hc0 = th_hi[ic0];
      lc0 = th_lo[ic0];
    }
    if (ic1 >= 0) {
      tc1 = theta[ic1];
      hc1 = th_hi[ic1];
      lc1 = th_lo[ic1];
    }
    for (int j = warp0; j < n; j += nwarps) {
      const int e0 = rowptr[j], e1 = rowptr[j + 1];
      T a0 = T(0), a1 = T(0);
      for (int eb = e0; eb < e1; eb += 32) {
        // the warp loads up to 32 (column, value) pairs, then broadcasts them
        const int e = eb + lane;
        int m = -1;
        T v = T(0);
        if (e < e1) {
          m = colind[e];
          v = ldval<T>(vals, e, v_dtype);
        }
        const int cnt = min(32, e1 - eb);
        for (int q = 0; q < cnt; ++q) {
          const int mq = __shfl_sync(0xffffffffu, m, q);
          const T vq = __shfl_sync(0xffffffffu, v, q);
          if (mq == j) continue;  // the diagonal is delta_j, applied below
          const V2 z = *reinterpret_cast<const V2*>(Zin + (int64_t)mq * kk + c0);
          a0 = fma(vq, z.x, a0);
          a1 = fma(vq, z.y, a1);
        }
      }
      const V2 zj = *reinterpret_cast<const V2*>(Zin + (int64_t)j * kk + c0);
      const T dj = (T)delta[j];
      const T p0 = fma(dj, zj.x, a0), p1 = fma(dj, zj.y, a1);
      T f0 = T(0), f1 = T(0), r0 = T(0), r1 = T(0);
      if (c0 < k) {
        T gap;
        if constexpr (sizeof(T) == 8) gap = theta[j] - tc0;
        else gap = gap2f(th_hi[j], th_lo[j], hc0, lc0);
        if (gap == T(0) && j != ic0) flag_degenerate(st);
        map_entry<T>(zj.x, p0, d0, gap, j == ic0, f0, r0);
        s_inc += (f0 - zj.x) * (f0 - zj.x);
        s_z += zj.x * zj.x;
        s_r += r0 * r0;
      }
      if (c1 < k) {
        T gap;
        if constexpr (sizeof(T) == 8) gap = theta[j] - tc1;
        else gap = gap2f(th_hi[j], th_lo[j], hc1, lc1);
        if (gap == T(0) && j != ic1) flag_degenerate(st);
        map_entry<T>(zj.y, p1, d1, gap, j == ic1, f1, r1);
        s_inc += (f1 - zj.y) * (f1 - zj.y);
        s_z += zj.y * zj.y;
        s_r += r1 * r1;
      }
      V2 fo;
      fo.x = f0;
      fo.y = f1;
      *reinterpret_cast<V2*>(Fout + (int64_t)j * kk + c0) = fo;
    }
  }
  const double b0 = warp_sum((double)s_inc), b1 = warp_sum((double)s_z),
               b2 = warp_sum((double)s_r);
  if (lane == 0) {
    atomicAdd(&st->acc_inc2, b0);
    atomicAdd(&st->acc_z2, b1);
    atomicAdd(&st->acc_r2, b2);
  }
}

// Row-major n x kk iterate -> column-major n x k output (ldo), 32x32 tiles.
template <typename TI, typename TO>
__global__ void k_csr_transpose_out(const TI* __restrict__ Z, int n, int k, int kk,
                                    TO* __restrict__ out, int64_t ldo) {
  __shared__ TI tile[32][33];
  const int j0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = 0; q < 32; q += 8) {
    const int j = j0 + ty + q, c = c0 + tx;
    tile[ty + q][tx] = (j < n && c < kk) ? Z[(int64_t)j * kk + c] : TI(0);
  }
  __syncthreads();
  for (int q = 0; q < 32; q += 8) {
    const int c = c0 + ty + q, j = j0 + tx;
    if (c < k && j < n) out[(int64_t)c * ldo + j] = (TO)tile[tx][ty + q];
  }
}

inline unsigned nblocks(int64_t total, int bs) { return (unsigned)((total + bs - 1) / bs); }

}  // namespace

// ---------------------------------------------------------------- launchers
void launch_csr_theta(const int32_t* rowptr, const int32_t* colind, const void* vals, int v_dtype,
                      const double* theta_in, int n, double* theta, float* th_hi, float* th_lo,
                      double* delta, DevState* st, cudaStream_t s) {
  k_csr_theta<<<nblocks((int64_t)n * 32, 256), 256, 0, s>>>(rowptr, colind, vals, v_dtype,
                                                            theta_in, n, theta, th_hi, th_lo,
                                                            delta, st);
}

void launch_csr_r0(const int32_t* rowptr, const int32_t* colind, const void* vals, int v_dtype,
                   int n, const int* count, double* part, int nblk, DevState* st,
                   cudaStream_t s) {
  k_csr_r0<<<nblk, 256, 0, s>>>(rowptr, colind, vals, v_dtype, n, count, part);
  k_csr_sum_r0<<<1, 256, 0, s>>>(part, nblk, st);
}

void launch_csr_init_z(const int32_t* icol, int n, int kk, void* Z, int f64, cudaStream_t s) {
  const unsigned g = nblocks((int64_t)n * kk, 256);
  if (f64) k_csr_init_z<double><<<g, 256, 0, s>>>(icol, n, kk, (double*)Z);
  else k_csr_init_z<float><<<g, 256, 0, s>>>(icol, n, kk, (float*)Z);
}

void launch_csr_prepass(const int32_t* rowptr, const int32_t* colind, const void* vals,
                        int v_dtype, const double* delta, const int32_t* icol, int kk,
                        const void* Z, int f64, double* d, DevState* st, cudaStream_t s) {
  const unsigned g = nblocks((int64_t)kk * 32, 256);
  if (f64)
    k_csr_prepass<double><<<g, 256, 0, s>>>(rowptr, colind, vals, v_dtype, delta, icol, kk,
                                            (const double*)Z, d, st);
  else
    k_csr_prepass<float><<<g, 256, 0, s>>>(rowptr, colind, vals, v_dtype, delta, icol, kk,
                                           (const float*)Z, d, st);
}

void launch_csr_spmm_map(const int32_t* rowptr, const int32_t* colind, const void* vals,
                         int v_dtype, const double* delta, const double* theta,
                         const float* th_hi, const float* th_lo, const int32_t* icol,
                         const double* d, int n, int k, int kk, const void* Zin, void* Fout,
                         int f64, int nblk, DevState* st, cudaStream_t s) {
  if (f64)
    k_csr_spmm_map<double><<<nblk, 256, 0, s>>>(rowptr, colind, vals, v_dtype, delta, theta,
                                                th_hi, th_lo, icol, d, n, k, kk,
                                                (const double*)Zin, (double*)Fout, st);
  else
    k_csr_spmm_map<float><<<nblk, 256, 0, s>>>(rowptr, colind, vals, v_dtype, delta, theta,
                                               th_hi, th_lo, icol, d, n, k, kk,
                                               (const float*)Zin, (float*)Fout, st);
}

void launch_csr_out(const void* Z, int f64, int n, int k, int kk, void* out, int64_t ldo,
                    int out_f64, cudaStream_t s) {
  dim3 g(nblocks(n, 32), nblocks(kk, 32)), b(32, 8);
  if (f64 && out_f64)
    k_csr_transpose_out<double, double><<<g, b, 0, s>>>((const double*)Z, n, k, kk,
                                                        (double*)out, ldo);
  else if (f64)
    k_csr_transpose_out<double, float><<<g, b, 0, s>>>((const double*)Z, n, k, kk, (float*)out,
                                                       ldo);
  else if (out_f64)
    k_csr_transpose_out<float, double><<<g, b, 0, s>>>((const float*)Z, n, k, kk, (double*)out,
                                                       ldo);
  else
    k_csr_transpose_out<float, float><<<g, b, 0, s>>>((const float*)Z, n, k, kk, (float*)out,
                                                      ldo);
}

}  // namespace ipt
