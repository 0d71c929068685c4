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
// Kernels: the diagonal pre-pass d_c = (Delta Z)_{cols[c], c} (one warp per
// column: a sparse row dot product; inside the SpMM for up to kFusedD
// columns), the SpMM + map, and the transpose of the result to the
// column-major output of the C ABI.  The setup pass over the rows
// and the FP64 residual are in k_csr_setup.cu.
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

// d_c = sum_m Delta_{i_c, m} Z_{m, c} = delta_{i_c} Z_{i_c, c} + sum over the
// off-diagonal stored entries of row i_c, by a group of 4 consecutive lanes
// (`sub` = lane & 3): each lane sums every 4th entry in storage order, the
// group adds its four sums pairwise (valid in every lane of the group).  Rows
// of the sparse workloads hold ~17 entries, so one dependent chain of loads
// per column, with 8 columns per warp in flight.
template <typename T>
__device__ __forceinline__ double csr_d_column(const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ colind,
                                               const void* __restrict__ vals, int v_dtype,
                                               const double* __restrict__ delta,
                                               const int32_t* __restrict__ icol, int kk,
                                               const T* __restrict__ Z, int c, int sub) {
  const int i = c < kk ? icol[c] : -1;
  double s = 0.0;
  if (i >= 0) {
    const int e1 = rowptr[i + 1];
    for (int e = rowptr[i] + sub; e < e1; e += 4) {
      const int m = colind[e];
      if (m != i) s += ldval<double>(vals, e, v_dtype) * (double)Z[(int64_t)m * kk + c];
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return i >= 0 ? s + delta[i] * (double)Z[(int64_t)i * kk + c] : 0.0;
}

// The pre-pass as its own launch (iterates wider than the SpMM's shared d):
// four lanes per column.
template <typename T>
__global__ void k_csr_prepass(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                              const void* __restrict__ vals, int v_dtype,
                              const double* __restrict__ delta, const int32_t* __restrict__ icol,
                              int kk, const T* __restrict__ Z, double* __restrict__ d,
                              const DevState* st) {
  if (st->done || (st->flags & FLAG_CSR_INDEX)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = t >> 2;  // whole warps stay in the loop (the group shuffles)
  const double v = csr_d_column<T>(rowptr, colind, vals, v_dtype, delta, icol, kk, Z, c, t & 3);
  if ((t & 3) == 0 && c < kk) d[c] = v;
}

// Widest iterate (kk columns) whose d the SpMM computes itself, in shared memory.
#ifndef IPT_CSR_FUSED_D
#define IPT_CSR_FUSED_D 512
#endif
constexpr int kFusedD = IPT_CSR_FUSED_D;

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
// With fuse_d (kk <= kFusedD) the kernel forms d itself: every CTA that
// evaluates a row computes all kk values into shared memory (four lanes per
// column, as the separate pre-pass does, so the values are the same), and the
// first CTA also stores them to d_out; otherwise d comes from the pre-pass.
template <typename T>
__global__ void __launch_bounds__(256, 4)
    k_csr_spmm_map(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                   const void* __restrict__ vals, int v_dtype, const double* __restrict__ delta,
                   const double* __restrict__ theta, const float* __restrict__ th_hi,
                   const float* __restrict__ th_lo, const int32_t* __restrict__ icol,
                   const double* __restrict__ d, double* __restrict__ d_out, int fuse_d, int n,
                   int k, int kk, const T* __restrict__ Zin, T* __restrict__ Fout,
                   DevState* st) {
  griddep_wait();  // launched with programmatic dependent launch in the loop
  griddep_launch();
  if (st->done || (st->flags & FLAG_CSR_INDEX)) return;
  using V4 = typename Four<T>::V;
  const int lane = threadIdx.x & 31, hl = lane & 15;
  const unsigned hmask = (lane < 16) ? 0x0000ffffu : 0xffff0000u;
  const int half0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 2 + (lane >> 4);
  const int nhalves = gridDim.x * (blockDim.x >> 5) * 2;
  const int wlo = st->win_lo, whi = st->win_hi;
  __shared__ double sd[kFusedD > 0 ? kFusedD : 1];
  if (fuse_d) {
    if (wlo + (int)blockIdx.x * (int)(blockDim.x >> 5) * 2 < whi || blockIdx.x == 0) {
      for (int c0 = 0; c0 < kk; c0 += (int)blockDim.x >> 2) {
        const int c = c0 + (threadIdx.x >> 2);
        const double v = csr_d_column<T>(rowptr, colind, vals, v_dtype, delta, icol, kk, Zin,
                                         c, threadIdx.x & 3);
        if ((threadIdx.x & 3) == 0 && c < kk) {
          sd[c] = v;
          if (blockIdx.x == 0) d_out[c] = v;
        }
      }
    }
    __syncthreads();
  }
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
      dc[u] = (T)(fuse_d ? sd[cb + u] : d[cb + u]);
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
  const int worked = __any_sync(0xffffffffu, wlo + half0 - (lane >> 4) < whi);
  // warp sums (FP32 pairs for FP32 iterates: FP64 adds run on the narrow FP64
  // pipe), skipped by the idle warps of the persistent grid
  double b0 = 0.0, b1 = 0.0, b2 = 0.0;
  if (worked) {
    if constexpr (sizeof(T) == 4) {
      b0 = f2_value(warp_sum(F2{(float)s_inc, 0.f}));
      b1 = f2_value(warp_sum(F2{(float)s_z, 0.f}));
      b2 = f2_value(warp_sum(F2{(float)s_r, 0.f}));
    } else {
      b0 = warp_sum((double)s_inc);
      b1 = warp_sum((double)s_z);
      b2 = warp_sum((double)s_r);
    }
  }
  f_lo = warp_min_int(f_lo);
  f_hi = warp_max_int(f_hi);
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
      if (rwork[q]) {
        t0 += red[0][q];
        t1 += red[1][q];
        t2 += red[2][q];
      }
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
void launch_csr_prepass(const int32_t* rowptr, const int32_t* colind, const void* vals,
                        int v_dtype, const double* delta, const int32_t* icol, int kk,
                        const void* Z, int f64, double* d, DevState* st, cudaStream_t s) {
  const unsigned g = nblocks((int64_t)kk * 4, 256);
  if (f64)
    k_csr_prepass<double><<<g, 256, 0, s>>>(rowptr, colind, vals, v_dtype, delta, icol, kk,
                                            (const double*)Z, d, st);
  else
    k_csr_prepass<float><<<g, 256, 0, s>>>(rowptr, colind, vals, v_dtype, delta, icol, kk,
                                           (const float*)Z, d, st);
}

int launch_csr_evaluate(const int32_t* rowptr, const int32_t* colind, const void* vals,
                        int v_dtype, const double* delta, const double* theta,
                        const float* th_hi, const float* th_lo, const int32_t* icol, double* d,
                        int n, int k, int kk, const void* Zin, void* Fout, int f64, int nblk,
                        DevState* st, cudaStream_t s, const cudaEvent_t* ev) {
  const int fuse = kk <= kFusedD ? 1 : 0;
  if (ev) cudaEventRecord(ev[0], s);
  if (!fuse) launch_csr_prepass(rowptr, colind, vals, v_dtype, delta, icol, kk, Zin, f64, d, st, s);
  if (ev) {
    cudaEventRecord(ev[1], s);
    cudaEventRecord(ev[2], s);
  }
  if (f64)
    launch_pdl(k_csr_spmm_map<double>, dim3(nblk), dim3(256), 0, s, rowptr, colind, vals,
               v_dtype, delta, theta, th_hi, th_lo, icol, (const double*)d, d, fuse, n, k, kk,
               (const double*)Zin, (double*)Fout, st);
  else
    launch_pdl(k_csr_spmm_map<float>, dim3(nblk), dim3(256), 0, s, rowptr, colind, vals,
               v_dtype, delta, theta, th_hi, th_lo, icol, (const double*)d, d, fuse, n, k, kk,
               (const float*)Zin, (float*)Fout, st);
  if (ev) cudaEventRecord(ev[3], s);
  return fuse ? 1 : 2;
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

}  // namespace ipt
