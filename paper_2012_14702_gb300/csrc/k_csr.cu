// Sparse IPT evaluation: P = Delta Z for M given in CSR (all stored entries of
// M, diagonal included), with the map of Eq. (dyn) fused into the same warp.
//
// Layout.  Internally Z is row-major n x kk (kk = k rounded up to 64), so the
// gather Z[m, :] of one column index m is a single coalesced 64-wide read
// (256 B in FP32).  In the SpMM a half-warp owns one row j of Delta at a time
// and lane l of the half the columns c = 64*chunk + 4l .. 4l+3 (one 16-byte
// gather per neighbour row).  The diagonal of Delta,
// delta_j = M_jj - theta_j (0 when theta = diag(M)), is applied separately, so
// the CSR loop skips stored diagonal entries.
//
// Kernels: setup (theta, delta_j, residual normaliser, Z = E), the diagonal
// pre-pass d_c = (Delta Z)_{cols[c], c} (one warp per column: a sparse row
// dot product), the SpMM + map, and the transpose of the result to the
// column-major output of the C ABI.
#include "ipt_internal.cuh"

#include <math.h>

#include <algorithm>

namespace ipt {

namespace {

template <typename T>
__device__ __forceinline__ T ldval(const void* v, int64_t i, int dt) {
  return dt == IPT_DTYPE_F64 ? (T) static_cast<const double*>(v)[i]
                             : (T) static_cast<const float*>(v)[i];
}

// One pass over the rows, a block per 256 consecutive rows [j0, j0 + 256):
// the block streams the stored entries of its rows, rowptr[j0] ..
// rowptr[j0 + 256], with consecutive threads on consecutive entries (the
// column-index and value reads are coalesced and all in flight at once; an
// entry's row is found by a binary search of the block's row bounds in shared
// memory).  Per row: the CSR structure check (row bounds within [0, nnz] and
// ascending, column indices in [0, n); a bad row is flagged, and the later CSR
// kernels then do nothing), the stored diagonal M_jj (0 if the row stores
// none; repeated diagonal entries add up, as in the product), theta_j (given,
// or M_jj), its FP32 split and delta_j = M_jj - theta_j; non-finite theta is
// flagged.  Per block: the partial of ||M Z0 - Z0 Lambda0||^2 (the squared
// off-diagonal entries in requested columns, count[col] > 0), the band
// max |j - m| of the stored entries and the row range of the requested rows
// (the support of Z0 = E).
__global__ void __launch_bounds__(256)
    k_csr_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
               const void* __restrict__ vals, int v_dtype, const double* __restrict__ theta_in,
               int n, int64_t nnz, const int* __restrict__ count, double* __restrict__ theta,
               float* __restrict__ th_hi, float* __restrict__ th_lo, double* __restrict__ delta,
               double* __restrict__ part, DevState* st) {
  __shared__ int sp[257];        // the block's row bounds, clamped to [0, nnz]
  __shared__ double sdiag[256];  // stored diagonal of each row
  const int t = threadIdx.x, j0 = blockIdx.x * 256;
  const int rows = min(256, n - j0);
  for (int i = t; i <= rows; i += 256)
    sp[i] = (int)min((int64_t)max(rowptr[j0 + i], 0), nnz);
  sdiag[t] = 0.0;
  float r0 = 0.f;
  int band = 0, lo = n, hi = -1;
  bool bad = false;
  if (t < rows) {
    const int j = j0 + t;
    const int e0 = rowptr[j], e1 = rowptr[j + 1];
    bad = !(e0 >= 0 && e0 <= e1 && (int64_t)e1 <= nnz && (j > 0 || e0 == 0) &&
            (j + 1 < n || (int64_t)e1 == nnz));
    if (count[j] > 0) lo = hi = j;
  }
  __syncthreads();
  const int eb = sp[0], ee = max(sp[rows], eb);
  // kU entries per thread per step, their loads (and then their gathers of
  // count[]) all issued before any is used
  constexpr int kU = 4;
  for (int e = eb + t; e < ee; e += 256 * kU) {
    int m[kU], cnt[kU];
    float v[kU];  // FP32: FP64 conversions run on the narrow FP64 pipe
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int x = e + 256 * u;
      m[u] = x < ee ? colind[x] : -1;
      v[u] = x < ee ? ldval<float>(vals, x, v_dtype) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) cnt[u] = (m[u] >= 0 && m[u] < n) ? count[m[u]] : 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int x = e + 256 * u;
      if (x >= ee) break;
      if (m[u] < 0 || m[u] >= n) {
        bad = true;
        continue;
      }
      // the entry's row: the last r with sp[r] <= x
      int a = 0, b = rows - 1;
      while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (sp[mid] <= x) a = mid;
        else b = mid - 1;
      }
      const int j = j0 + a;
      band = max(band, abs(m[u] - j));
      if (m[u] == j) {
        atomicAdd(&sdiag[a], ldval<double>(vals, x, v_dtype));  // once per row
      } else if (cnt[u] > 0) {
        r0 = fmaf(v[u], v[u], r0);
      }
    }
  }
  __syncthreads();
  if (bad) atomicOr(&st->flags, FLAG_CSR_INDEX);
  if (t < rows) {
    const int j = j0 + t;
    const double mjj = sdiag[t];
    const double th = theta_in ? theta_in[j] : mjj;
    if (!isfinite(th)) atomicOr(&st->flags, FLAG_THETA_NONFINITE);
    theta[j] = th;
    const float h = (float)th;
    th_hi[j] = h;
    th_lo[j] = (float)(th - (double)h);
    delta[j] = mjj - th;
    reinterpret_cast<float*>(delta + n)[j] = (float)(mjj - th);  // FP32 copy for FP32 kernels
  }
  // block reduction; the shared words take one atomic per block, and only
  // when the block's value would change them (most blocks see the same band)
  __shared__ float red[8];
  __shared__ int rb[8], rl[8], rh[8];
  const int wq = threadIdx.x >> 5;
  const float w = warp_sum(r0);
  band = warp_max_int(band);
  lo = warp_min_int(lo);
  hi = warp_max_int(hi);
  if ((threadIdx.x & 31) == 0) {
    red[wq] = w;
    rb[wq] = band;
    rl[wq] = lo;
    rh[wq] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    int b = 0, l = n, hh = -1;
    for (int q = 0; q < 8; ++q) {
      tot += (double)red[q];
      b = max(b, rb[q]);
      l = min(l, rl[q]);
      hh = max(hh, rh[q]);
    }
    part[blockIdx.x] = tot;
    if (b > *(volatile int*)&st->band) atomicMax(&st->band, b);
    if (hh >= 0) {
      atomicMin(&st->z_lo, l);
      atomicMax(&st->z_hi, hh);
    }
  }
}

// One block: ||R0||^2 from the row pass's partials, and the rows the first
// product evaluates: all of them, or (window) the requested rows widened by
// the band (rows further away have no stored entry in a nonzero row of E).
__global__ void __launch_bounds__(1024)
    k_csr_sum_r0(const double* __restrict__ part, int count, int n, int window, DevState* st) {
  __shared__ double red[1024];
  double t = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) t += part[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->r0acc = red[0];
    st->nz_lo = n;
    st->nz_hi = -1;
    if (window && st->z_hi >= st->z_lo) {
      st->win_lo = max(0, st->z_lo - st->band);
      st->win_hi = (int)min((int64_t)n, (int64_t)st->z_hi + 1 + st->band);
    } else {
      st->win_lo = 0;
      st->win_hi = n;
    }
  }
}

// Z = E in the row-major layout (Z[j*kk + c] = 1 at j = cols[c]); padding
// zero.  Block: 64 columns x 4 rows; each thread writes one entry per row step.
template <typename T>
__global__ void k_csr_units(const int32_t* __restrict__ icol, int k, int kk, T* __restrict__ Z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int i = icol[c];  // -1 for a column index out of range (flagged)
  if (i >= 0) Z[(int64_t)i * kk + c] = T(1);
}

// d_c = sum_m Delta_{i_c, m} Z_{m, c} = delta_{i_c} Z_{i_c, c} + sum over the
// off-diagonal stored entries of row i_c.  One warp per column.
template <typename T>
__global__ void k_csr_prepass(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                              const void* __restrict__ vals, int v_dtype,
                              const double* __restrict__ delta, const int32_t* __restrict__ icol,
                              int kk, const T* __restrict__ Z, double* __restrict__ d,
                              const DevState* st) {
  if (st->done || (st->flags & FLAG_CSR_INDEX)) return;
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

template <typename T>
struct Four;
template <>
struct Four<float> {
  using V = float4;
};
template <>
struct Four<double> {
  using V = double4;
};

// SpMM + map.  Persistent: a grid of CTAs of 8 warps walks the rows; each
// half-warp owns one row at a time (two independent rows per warp, so two
// rowptr -> colind -> gather chains are in flight), lane l of the half owns
// the 4 columns 64*chunk + 4l .. 4l+3 and gathers them as one 16-byte vector.
// The half loads up to 16 (column, value) pairs at once and broadcasts them
// with width-16 shuffles; the stored diagonal gets weight 0 (delta_j is
// applied in the epilogue).  Only rows [win_lo, win_hi) are evaluated (all
// rows unless the active window is on); the row range of the nonzero rows of
// F is recorded for the next window.  Norm partials: one atomic per warp.
template <typename T>
__global__ void __launch_bounds__(256, 4)
    k_csr_spmm_map(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                   const void* __restrict__ vals, int v_dtype, const double* __restrict__ delta,
                   const double* __restrict__ theta, const float* __restrict__ th_hi,
                   const float* __restrict__ th_lo, const int32_t* __restrict__ icol,
                   const double* __restrict__ d, int n, int k, int kk, const T* __restrict__ Zin,
                   T* __restrict__ Fout, DevState* st) {
  if (st->done || (st->flags & FLAG_CSR_INDEX)) return;
  using V4 = typename Four<T>::V;
  const int lane = threadIdx.x & 31, hl = lane & 15;
  const unsigned hmask = (lane < 16) ? 0x0000ffffu : 0xffff0000u;
  const int half0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 2 + (lane >> 4);
  const int nhalves = gridDim.x * (blockDim.x >> 5) * 2;
  const int wlo = st->win_lo, whi = st->win_hi;
  T s_inc = T(0), s_z = T(0), s_r = T(0);
  int f_lo = n, f_hi = -1;
  for (int ch = 0; ch < kk; ch += 64) {
    const int cb = ch + 4 * hl;
    int ic[4];
    T dc[4];
    double tc[4];
    float hc[4], lc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ic[u] = icol[cb + u];
      dc[u] = (T)d[cb + u];
      tc[u] = ic[u] >= 0 ? theta[ic[u]] : 0.0;
      hc[u] = ic[u] >= 0 ? th_hi[ic[u]] : 0.f;
      lc[u] = ic[u] >= 0 ? th_lo[ic[u]] : 0.f;
    }
    // both halves of a warp iterate together; a half past the last row idles
    for (int jb = wlo + half0 - (lane >> 4); jb < whi; jb += nhalves) {
      const int j = jb + (lane >> 4);
      const bool live = j < whi;
      const int e0 = live ? rowptr[j] : 0, e1 = live ? rowptr[j + 1] : 0;
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (int eb = e0; eb < e1; eb += 16) {
        const int e = eb + hl;
        int m = j;
        T v = T(0);
        if (e < e1) {
          m = colind[e];
          v = m == j ? T(0) : ldval<T>(vals, e, v_dtype);
        }
        const int cnt = min(16, e1 - eb);
        // four gathers in flight at a time (entries past the row's end are
        // (row j, weight 0): valid addresses that add nothing); the sums keep
        // the entry order
        for (int q = 0; q < cnt; q += 4) {
          int mq[4];
          T vq[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            mq[u] = __shfl_sync(hmask, m, q + u, 16);
            vq[u] = __shfl_sync(hmask, v, q + u, 16);
          }
          V4 z[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            z[u] = *reinterpret_cast<const V4*>(Zin + (int64_t)mq[u] * kk + cb);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            acc[0] = fma(vq[u], z[u].x, acc[0]);
            acc[1] = fma(vq[u], z[u].y, acc[1]);
            acc[2] = fma(vq[u], z[u].z, acc[2]);
            acc[3] = fma(vq[u], z[u].w, acc[3]);
          }
        }
      }
      if (!live) continue;
      const V4 zj4 = *reinterpret_cast<const V4*>(Zin + (int64_t)j * kk + cb);
      const T zj[4] = {zj4.x, zj4.y, zj4.z, zj4.w};
      T dj;  // no per-row FP64 conversion in the FP32 kernel
      if constexpr (sizeof(T) == 8) dj = delta[j];
      else dj = reinterpret_cast<const float*>(delta + n)[j];
      const float hj = th_hi[j], lj = th_lo[j];
      T fo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        fo[u] = T(0);
        if (cb + u < k) {
          const T p = fma(dj, zj[u], acc[u]);
          T gap;
          if constexpr (sizeof(T) == 8) gap = theta[j] - tc[u];
          else gap = gap2f(hj, lj, hc[u], lc[u]);
          if (gap == T(0) && j != ic[u]) flag_degenerate(st);
          T f, r;
          map_entry<T>(zj[u], p, dc[u], gap, j == ic[u], f, r);
          fo[u] = f;
          if (f != T(0)) {
            f_lo = min(f_lo, j);
            f_hi = max(f_hi, j);
          }
          s_inc += (f - zj[u]) * (f - zj[u]);
          s_z += zj[u] * zj[u];
          s_r += r * r;
        }
      }
      V4 out;
      out.x = fo[0];
      out.y = fo[1];
      out.z = fo[2];
      out.w = fo[3];
      *reinterpret_cast<V4*>(Fout + (int64_t)j * kk + cb) = out;
    }
  }
  // one set of atomics per block that evaluated a row (they all hit the same
  // few words, so idle blocks of the persistent grid must not add any)
  __shared__ double red[3][8];
  __shared__ int rlo[8], rhi[8], rwork[8];
  const int w = threadIdx.x >> 5;
  const double b0 = warp_sum((double)s_inc), b1 = warp_sum((double)s_z),
               b2 = warp_sum((double)s_r);
  f_lo = warp_min_int(f_lo);
  f_hi = warp_max_int(f_hi);
  const int worked = __any_sync(0xffffffffu, wlo + half0 - (lane >> 4) < whi);
  if (lane == 0) {
    red[0][w] = b0;
    red[1][w] = b1;
    red[2][w] = b2;
    rlo[w] = f_lo;
    rhi[w] = f_hi;
    rwork[w] = worked;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    int lo = n, hi = -1, any = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      t0 += red[0][q];
      t1 += red[1][q];
      t2 += red[2][q];
      lo = min(lo, rlo[q]);
      hi = max(hi, rhi[q]);
      any |= rwork[q];
    }
    if (any) {
      atomicAdd(&st->acc_inc2, t0);
      atomicAdd(&st->acc_z2, t1);
      atomicAdd(&st->acc_r2, t2);
    }
    if (hi >= 0) {
      atomicMin(&st->nz_lo, lo);
      atomicMax(&st->nz_hi, hi);
    }
  }
}

// Rows [j_lo, n) of the row-major n x kk iterate -> column-major n x k output
// (ldo), 32x32 tiles.
template <typename TI, typename TO>
__global__ void k_csr_transpose_out(const TI* __restrict__ Z, int j_lo, int n, int k, int kk,
                                    TO* __restrict__ out, int64_t ldo) {
  __shared__ TI tile[32][33];
  const int j0 = j_lo + blockIdx.x * 32, c0 = blockIdx.y * 32;
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
void launch_csr_rows(const int32_t* rowptr, const int32_t* colind, const void* vals, int v_dtype,
                     const double* theta_in, int n, int64_t nnz, const int* count, double* theta,
                     float* th_hi, float* th_lo, double* delta, double* part, int window,
                     DevState* st, cudaStream_t s) {
  const unsigned g = nblocks(n, 256);  // one block per 256 rows (the partials' capacity)
  k_csr_rows<<<g, 256, 0, s>>>(rowptr, colind, vals, v_dtype, theta_in, n, nnz, count, theta, th_hi,
                               th_lo, delta, part, st);
  k_csr_sum_r0<<<1, 1024, 0, s>>>(part, (int)g, n, window, st);
}

void launch_csr_units(const int32_t* icol, int k, int kk, void* Z, int f64, cudaStream_t s) {
  if (f64) k_csr_units<double><<<nblocks(k, 256), 256, 0, s>>>(icol, k, kk, (double*)Z);
  else k_csr_units<float><<<nblocks(k, 256), 256, 0, s>>>(icol, k, kk, (float*)Z);
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

void launch_csr_out(const void* Z, int f64, int j_lo, int n, int k, int kk, void* out,
                    int64_t ldo, int out_f64, cudaStream_t s) {
  if (n <= j_lo) return;
  dim3 g(nblocks(n - j_lo, 32), nblocks(kk, 32)), b(32, 8);
  if (f64 && out_f64)
    k_csr_transpose_out<double, double><<<g, b, 0, s>>>((const double*)Z, j_lo, n, k,
                                                        kk, (double*)out, ldo);
  else if (f64)
    k_csr_transpose_out<double, float><<<g, b, 0, s>>>((const double*)Z, j_lo, n, k, kk,
                                                       (float*)out, ldo);
  else if (out_f64)
    k_csr_transpose_out<float, double><<<g, b, 0, s>>>((const float*)Z, j_lo, n, k, kk,
                                                       (double*)out, ldo);
  else
    k_csr_transpose_out<float, float><<<g, b, 0, s>>>((const float*)Z, j_lo, n, k, kk,
                                                      (float*)out, ldo);
}

namespace {

// ||M Z - Z Lambda||_F^2 in FP64 (verification of a sparse result): the stored
// entries of M (diagonal included) against the row-major iterate; one warp per
// row, lane l the columns c = c0 + l of each 32-column chunk.
template <typename T>
__global__ void __launch_bounds__(256)
    k_csr_residual64(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                     const void* __restrict__ vals, int v_dtype, int n, int k, int kk,
                     const T* __restrict__ Z, const double* __restrict__ lam,
                     double* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s = 0.0;
  for (int64_t j = w0; j < n; j += nw) {
    const int e0 = rowptr[j], e1 = rowptr[j + 1];
    for (int c0 = 0; c0 < k; c0 += 32) {
      const int c = c0 + lane;
      if (c >= k) continue;
      double a = 0.0;
      for (int e = e0; e < e1; ++e) {
        const double v = v_dtype == IPT_DTYPE_F64 ? static_cast<const double*>(vals)[e]
                                                  : (double)static_cast<const float*>(vals)[e];
        a = fma(v, (double)Z[(int64_t)colind[e] * kk + c], a);
      }
      const double r = a - (double)Z[j * kk + c] * lam[c];
      s += r * r;
    }
  }
  s = warp_sum(s);
  if (lane == 0) atomicAdd(acc, s);
}

}  // namespace

void launch_csr_residual64(const int32_t* rowptr, const int32_t* colind, const void* vals,
                           int v_dtype, int n, int k, int kk, const void* Z, int f64,
                           const double* lam, double* acc, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(((int64_t)n + 7) / 8, 152 * 16);
  if (f64)
    k_csr_residual64<double><<<blocks, 256, 0, s>>>(rowptr, colind, vals, v_dtype, n, k, kk,
                                                    (const double*)Z, lam, acc);
  else
    k_csr_residual64<float><<<blocks, 256, 0, s>>>(rowptr, colind, vals, v_dtype, n, k, kk,
                                                   (const float*)Z, lam, acc);
}

}  // namespace ipt
