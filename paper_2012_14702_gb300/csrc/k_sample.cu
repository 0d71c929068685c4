// Sampled error of a tensor-core product P ~ Delta Z.
//
// The split 16-bit products accumulate in the tensor core's FP32 accumulators,
// whose rounding depends on how each sum grows; an a-priori bound on it is far
// from the error actually made.  Instead, at the evaluations whose error
// matters (a re-base, a possible last evaluation), the product's epilogue keeps
// P at kSampleRows fixed rows j_r = r * stride + off, and this kernel
// recomputes those entries from the same FP32 iterate Z: the sum
// sum_m Delta_{j m} W_{m c} over W = Z - E with compensated FP32 sums (FP32
// partials of 32 products added into TwoSum pairs, as the compensated FP32
// product does), plus Delta_{j, cols[c]} exactly.  The squared differences over
// the sampled entries, scaled by the entries of P over the entries sampled,
// estimate ||P - Delta Z||_F^2 (k_control), which enters the residual
// R = M Z - Z Lambda one to one.
//
// Shape: a CTA owns SC = 32 columns; its 256 threads are 8 row groups of 32
// (thread = one column, two sampled rows).  At most kMaxBlocks column blocks,
// spread evenly over the columns, are sampled (k <= 2048: all of them).  Rows
// of Z come in chunks of 128 through shared memory as 16-byte loads, the next
// chunk's loads issued into registers before the current chunk's products.
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int SC = 32;               // columns per CTA
constexpr int SK = 128;              // rows of Z per shared-memory chunk
constexpr int SR = kSampleRows;      // sampled rows
constexpr int RPT = SR / 8;          // sampled rows per thread (8 groups of 32 threads)
constexpr int PART = 32;             // products per FP32 partial
constexpr int kMaxBlocks = 64;       // column blocks sampled at most
constexpr int ZV = SC * SK / 4 / 256;  // float4 loads of Z per thread and chunk
constexpr int DV = SR * SK / 4 / 256;  // float4 loads of Delta per thread and chunk
static_assert(ZV * 256 * 4 == SC * SK && DV * 256 * 4 == SR * SK, "load split");

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bv = __fsub_rn(s, hi);
  const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(x, bv));
  hi = s;
  lo = __fadd_rn(lo, er);
}

__global__ void __launch_bounds__(256)
    k_sample_exact(const float* __restrict__ Drow, const float* __restrict__ Z,
                   const int32_t* __restrict__ icol, int n, int k, int kpad, int64_t ld,
                   const float* __restrict__ psmp, int stride, int off, DevState* st, DynZ dz) {
  if (st->done) return;
  if (dz.dyn) {
    if (st->pause || !st->measure) return;
    Z = dz.z[st->cur];
  }
  __shared__ float Zs[SK][SC + 1];
  __shared__ float Ds[SR][SK + 4];
  __shared__ int sic[SC];
  __shared__ double red[8][2];
  const int tid = threadIdx.x, cl = tid & (SC - 1), rg = tid >> 5;
  const int nblk = kpad / SC;
  const int c0 = (int)(((int64_t)blockIdx.x * nblk) / gridDim.x) * SC;
  if (tid < SC) sic[tid] = (c0 + tid < k) ? icol[c0 + tid] : -1;
  __syncthreads();
  // this thread's load slots: Z float4 f = tid + 256 q -> column f / (SK/4),
  // rows 4 (f % (SK/4)); Delta float4 f -> sampled row f / (SK/4), columns
  // 4 (f % (SK/4))
  float4 zr[ZV], dr[DV];
  auto load = [&](int64_t m0) {
#pragma unroll
    for (int q = 0; q < ZV; ++q) {
      const int f = tid + 256 * q, cc = f / (SK / 4), m4 = f % (SK / 4);
      zr[q] = sic[cc] >= 0
                  ? *reinterpret_cast<const float4*>(Z + (int64_t)(c0 + cc) * ld + m0 +
                                                     4 * m4)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < DV; ++q) {
      const int f = tid + 256 * q, r = f / (SK / 4), m4 = f % (SK / 4);
      const int j = r * stride + off;
      dr[q] = j < n ? *reinterpret_cast<const float4*>(Drow + (int64_t)j * ld + m0 + 4 * m4)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stash = [&](int64_t m0) {
#pragma unroll
    for (int q = 0; q < ZV; ++q) {
      const int f = tid + 256 * q, cc = f / (SK / 4), m4 = f % (SK / 4);
      const int ic = sic[cc];
      float v[4] = {zr[q].x, zr[q].y, zr[q].z, zr[q].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t m = m0 + 4 * m4 + u;
        Zs[4 * m4 + u][cc] = v[u] - (m == ic ? 1.f : 0.f);  // W = Z - E
      }
    }
#pragma unroll
    for (int q = 0; q < DV; ++q) {
      const int f = tid + 256 * q, r = f / (SK / 4), m4 = f % (SK / 4);
      *reinterpret_cast<float4*>(&Ds[r][4 * m4]) = dr[q];
    }
  };
  float acc[RPT], hi[RPT], lo[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) acc[q] = hi[q] = lo[q] = 0.f;
  load(0);
  for (int64_t m0 = 0; m0 < ld; m0 += SK) {
    stash(m0);
    __syncthreads();
    if (m0 + SK < ld) load(m0 + SK);  // in flight during this chunk's products
#pragma unroll 1
    for (int p0 = 0; p0 < SK; p0 += PART) {
#pragma unroll 8
      for (int mm = p0; mm < p0 + PART; ++mm) {
        const float w = Zs[mm][cl];
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q] = fmaf(Ds[rg * RPT + q][mm], w, acc[q]);
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        two_sum_add(hi[q], lo[q], acc[q]);
        acc[q] = 0.f;
      }
    }
    __syncthreads();
  }
  double sum = 0.0, cnt = 0.0;
  const int c = c0 + cl, ic = sic[cl];
  if (ic >= 0) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = rg * RPT + q, j = r * stride + off;
      if (j >= n || j == ic) continue;  // the unit entry's P is not used by the map
      const double exact = (double)hi[q] + (double)lo[q] + (double)Drow[(int64_t)j * ld + ic];
      const double dlt = (double)psmp[(int64_t)r * kpad + c] - exact;
      sum += dlt * dlt;
      cnt += 1.0;
    }
  }
  sum = warp_sum(sum);
  cnt = warp_sum(cnt);
  if ((tid & 31) == 0) {
    red[tid >> 5][0] = sum;
    red[tid >> 5][1] = cnt;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0, u = 0.0;
    for (int w = 0; w < 8; ++w) {
      t += red[w][0];
      u += red[w][1];
    }
    atomicAdd(&st->acc_dp2, t);
    atomicAdd(&st->acc_dpn, u);
  }
}

}  // namespace

void launch_sample_exact(const float* Drow, const float* Z, const int32_t* icol, int n, int k,
                         int kpad, int64_t ld, const float* psmp, int stride, int off,
                         DevState* st, const DynZ& dz, cudaStream_t s) {
  const int blocks = kpad / SC < kMaxBlocks ? kpad / SC : kMaxBlocks;
  k_sample_exact<<<(unsigned)blocks, 256, 0, s>>>(Drow, Z, icol, n, k, kpad, ld, psmp, stride,
                                                  off, st, dz);
}

}  // namespace ipt
