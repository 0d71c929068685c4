// Sparse IPT, the kernels outside the evaluation loop: the one setup pass over
// the rows of M (CSR structure check, theta, delta_j = M_jj - theta_j, the
// residual normaliser ||M Z0 - Z0 Lambda0|| and the band; the support of
// Z0 = E and its unit entries come from the column validation), and the FP64
// residual ||M Z - Z Lambda||_F that verifies a result.
#include "ipt_internal.cuh"

#include <limits.h>
#include <math.h>

#include <algorithm>

namespace ipt {

namespace {

inline unsigned nblocks(int64_t total, int bs) { return (unsigned)((total + bs - 1) / bs); }

// The per-row values of the row pass with plain FP64 arithmetic, for the rows
// the integer conversions do not cover (repeated diagonal entries of FP32
// input, values outside FP32's normal range).  Out of line, so that the common
// path issues no FP64-pipe instructions.  The stored diagonal: the first entry
// as stored, later ones (repeated entries) added in FP64 in storage order.
struct RowValues {
  double mjj, th, dj;
  float h, l, d;
};
__device__ __noinline__ RowValues csr_row_values_slow(const int32_t* __restrict__ colind,
                                                      const void* __restrict__ vals,
                                                      int v_dtype, int j, int e0, int e1,
                                                      const double* __restrict__ theta_in,
                                                      double mjj) {
  if (v_dtype != IPT_DTYPE_F64) {
    const float* v32 = static_cast<const float*>(vals);
    double first = 0.0, rest = 0.0;
    bool seen = false;
    for (int x = e0; x < e1; ++x) {
      if (colind[x] != j) continue;
      if (seen) rest += (double)v32[x];
      else first = (double)v32[x];
      seen = true;
    }
    mjj = first + rest;
  }
  RowValues r;
  r.mjj = mjj;
  r.th = theta_in ? theta_in[j] : mjj;
  r.h = (float)r.th;
  r.l = (float)(r.th - (double)r.h);
  r.dj = theta_in ? mjj - r.th : 0.0;
  r.d = (float)r.dj;
  return r;
}

// One pass over the rows, a block per 256 consecutive rows, a warp per 32 of
// them: the warp copies its rows' stored entries (one contiguous range of the
// CSR arrays) into shared memory in chunks with coalesced loads, then each lane
// walks its own row there, keeping the row's smallest and largest column
// index (its bounds check and its band).  Per row: the CSR structure check
// (row bounds within [0, nnz] and ascending, column indices in [0, n); a bad
// row is flagged, and the later CSR kernels then do nothing), the stored
// diagonal M_jj (0 if the row stores
// none; repeated diagonal entries add up, as in the product), theta_j (given,
// or M_jj), its FP32 split and delta_j = M_jj - theta_j; non-finite theta is
// flagged.  Per block: the partial of ||M Z0 - Z0 Lambda0||^2 (the squared
// off-diagonal entries in requested columns, count[col] > 0) and the band
// max |j - m| of the stored entries.  The requested columns' range
// [z_lo, z_hi] (set by the column validation before this pass) filters the
// count[] gathers: an entry outside it is in no requested column.
__global__ void __launch_bounds__(256, 4)
    k_csr_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
               const void* __restrict__ vals, int v_dtype, const double* __restrict__ theta_in,
               int n, int64_t nnz, const int* __restrict__ count, double* __restrict__ theta,
               float* __restrict__ th_hi, float* __restrict__ th_lo, double* __restrict__ delta,
               double* __restrict__ part, DevState* st) {
  constexpr int kW = 512;  // entries per warp chunk
  __shared__ int scol[8][kW];
  __shared__ float sval[8][kW];  // FP32 input only
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int j = blockIdx.x * 256 + threadIdx.x;  // this lane's row
  const bool live = j < n;
  const bool f64in = v_dtype == IPT_DTYPE_F64;
  float r0 = 0.f;
  int band = 0;
  bool bad = false;
  // requested columns: [clo, chi] (none if chi < clo)
  const int clo = st->z_lo, chi = st->z_hi;
  const bool anyreq = chi >= clo;
  const unsigned span = (unsigned)(chi - clo);
  int e0 = 0, e1 = 0;  // the row's entries, clamped to [0, nnz]
  if (live) {
    if (count[j] > 1) atomicOr(&st->flags, FLAG_COL_DUP);  // a column requested twice
    const int r0p = rowptr[j], r1p = rowptr[j + 1];
    bad = !(r0p >= 0 && r0p <= r1p && (int64_t)r1p <= nnz && (j > 0 || r0p == 0) &&
            (j + 1 < n || (int64_t)r1p == nnz));
    e0 = (int)min((int64_t)max(r0p, 0), nnz);
    e1 = max(e0, (int)min((int64_t)max(r1p, 0), nnz));
  }
  // the warp's range: from its first live row's start to its last live row's end
  const unsigned live_mask = __ballot_sync(0xffffffffu, live);
  int E0 = e0, E1 = e1;
  E0 = __shfl_sync(0xffffffffu, E0, live_mask ? __ffs(live_mask) - 1 : 0);
  E1 = __shfl_sync(0xffffffffu, E1, live_mask ? 31 - __clz(live_mask) : 0);
  E1 = max(E1, E0);
  // per row: the smallest and largest column index (bounds and band), and the
  // stored diagonal: FP64 input summed in FP64; FP32 input's first entry
  int mmin = INT_MAX, mmax = INT_MIN, ndiag = 0;
  float d32 = 0.f;
  double d64 = 0.0;
  for (int cs = E0; cs < E1; cs += kW) {
    const int ce = min(cs + kW, E1);
    __syncwarp();
    // all of the chunk's loads of a lane (kW / 32 of each array) in flight before
    // its shared-memory stores; FP64 values stay in global memory (read for the
    // diagonal and the requested columns only)
    constexpr int kPer = kW / 32;
    int cv[kPer];
    float vv[kPer];
    const float* v32 = static_cast<const float*>(vals);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int x = cs + lane + 32 * q;
      cv[q] = x < ce ? colind[x] : 0;
      vv[q] = (!f64in && x < ce) ? v32[x] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      scol[wq][lane + 32 * q] = cv[q];
      if (!f64in) sval[wq][lane + 32 * q] = vv[q];
    }
    __syncwarp();
    const int xb = max(e0, cs), xe = min(e1, ce);
#pragma unroll 4
    for (int x = xb; x < xe; ++x) {
      const int m = scol[wq][x - cs];
      mmin = min(mmin, m);
      mmax = max(mmax, m);
      // count[] only inside the requested columns' range (so also inside [0, n))
      const int cm = (anyreq && (unsigned)(m - clo) <= span) ? count[m] : 0;
      if (m == j) {
        if (f64in) d64 += static_cast<const double*>(vals)[x];
        else if (ndiag == 0) d32 = sval[wq][x - cs];
        ++ndiag;
      } else if (cm > 0) {
        const float v = f64in ? (float)static_cast<const double*>(vals)[x] : sval[wq][x - cs];
        r0 = fmaf(v, v, r0);
      }
    }
  }
  if (live && e1 > e0) {
    if (mmin < 0 || mmax >= n) bad = true;
    else band = max(j - mmin, mmax - j);
  }
  if (bad) atomicOr(&st->flags, FLAG_CSR_INDEX);
  if (live) {
    // the FP32 <-> FP64 conversions go through the integer ALU (the FP64 pipe
    // is narrow); only a given theta costs one FP64 subtraction per row, and
    // the rare rows the integer forms do not cover take the out-of-line path
    bool ok = true, ok1;
    double mjj = d64;
    if (v_dtype != IPT_DTYPE_F64 && ndiag > 0) {
      mjj = f32_to_f64_bits(d32, ok1);
      ok = ok1 && ndiag == 1;
    }
    double th = theta_in ? theta_in[j] : mjj;
    float h, l;
    split_f64_bits(th, h, l, ok1);
    ok = ok && ok1;
    double dj = theta_in ? mjj - th : 0.0;  // theta = M_jj exactly otherwise
    float d = f64_to_f32_rn_bits(dj, ok1);
    ok = ok && ok1;
    if (!ok) {
      const RowValues r = csr_row_values_slow(colind, vals, v_dtype, j, e0, e1, theta_in, mjj);
      th = r.th;
      h = r.h;
      l = r.l;
      dj = r.dj;
      d = r.d;
    }
    const unsigned long long tb = (unsigned long long)__double_as_longlong(th);
    if (((tb >> 52) & 0x7ffu) == 0x7ffu) atomicOr(&st->flags, FLAG_THETA_NONFINITE);
    theta[j] = th;
    th_hi[j] = h;
    th_lo[j] = l;
    delta[j] = dj;
    reinterpret_cast<float*>(delta + n)[j] = d;  // FP32 copy for FP32 kernels
  }
  // block reduction; the band takes one atomic per block, and only when the
  // block's value would change it (most blocks see the same band)
  __shared__ float red[8];
  __shared__ int rb[8];
  const float w = warp_sum(r0);
  band = warp_max_int(band);
  if ((threadIdx.x & 31) == 0) {
    red[wq] = w;
    rb[wq] = band;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    int b = 0;
    for (int q = 0; q < 8; ++q) {
      tot += (double)red[q];
      b = max(b, rb[q]);
    }
    part[blockIdx.x] = tot;
    if (b > *(volatile int*)&st->band) atomicMax(&st->band, b);
  }
}

// One block: ||R0||^2 from the row pass's partials (a fixed order), and the
// rows the first product evaluates: all of them, or (window) the requested
// rows widened by the band (rows further away have no stored entry in a
// nonzero row of E).  Launched with programmatic dependent launch after the
// row pass (a last-block reduction inside the row pass, measured, cost every
// block a memory fence: 63 -> 77 us).
__global__ void __launch_bounds__(1024)
    k_csr_sum_r0(const double* __restrict__ part, int count, int n, int window, DevState* st) {
  griddep_wait();
  griddep_launch();
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

}  // namespace

void launch_csr_rows(const int32_t* rowptr, const int32_t* colind, const void* vals, int v_dtype,
                     const double* theta_in, int n, int64_t nnz, const int* count, double* theta,
                     float* th_hi, float* th_lo, double* delta, double* part, int window,
                     DevState* st, cudaStream_t s) {
  const unsigned g = nblocks(n, 256);  // one block per 256 rows (the partials' capacity)
  k_csr_rows<<<g, 256, 0, s>>>(rowptr, colind, vals, v_dtype, theta_in, n, nnz, count, theta, th_hi,
                               th_lo, delta, part, st);
  launch_pdl(k_csr_sum_r0, dim3(1), dim3(1024), 0, s, (const double*)part, (int)g, n, window, st);
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
