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
// Shape: a CTA owns SC = 32 columns; its 256 threads are 32 columns x 8
// K-groups (a warp per K-group), and each thread keeps all 16 sampled rows of
// its column in registers, so one shared-memory read of Z feeds 16 products
// (the 16 entries of Delta at that K index are four broadcast 16-byte reads).
// At most kMaxBlocks column blocks, spread evenly over the columns, are sampled.
// Rows of Z come in chunks of 128 through shared memory as 16-byte loads, the
// next chunk's loads issued into registers before the current chunk's
// products; each chunk's 16 products per row form one FP32 partial.  The
// K-groups' pairs are added in group order in FP64 at the end.
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int SC = 32;               // columns per CTA
constexpr int SK = 128;              // rows of Z per shared-memory chunk
constexpr int SR = kSampleRows;      // sampled rows
constexpr int KG = 8;                // K-groups (warps)
constexpr int kMaxBlocks = 32;       // column blocks sampled at most
constexpr int KS = 4;                // K ranges per column block (one CTA each)
constexpr int ZV = SC * SK / 4 / 256;  // float4 loads of Z per thread and chunk
constexpr int DV = SR * SK / 4 / 256;  // float4 loads of Delta per thread and chunk
static_assert(ZV * 256 * 4 == SC * SK && DV * 256 * 4 == SR * SK, "load split");
static_assert(SR == 16, "four 16-byte reads of Delta per K index");

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
                   const float* __restrict__ psmp, int stride, int off, double* __restrict__ part,
                   int* __restrict__ arrived, DevState* st, DynZ dz) {
  griddep_wait();  // launched with programmatic dependent launch
  griddep_launch();
  if (st->done) return;
  if (dz.dyn) {
    if (st->pause || !st->measure) return;
    Z = dz.z[st->cur];
  }
  // CTA = (column block cb, K range ks): rows [k0, k1) of Z, chunk-aligned
  const int cb = blockIdx.x / KS, ks = blockIdx.x % KS, ncb = gridDim.x / KS;
  const int64_t nchunks = ld / SK;
  const int64_t k0 = (nchunks * ks / KS) * SK, k1 = (nchunks * (ks + 1) / KS) * SK;
  __shared__ union Smem {
    struct {
      float Zs[SK][SC + 1];
      float4 Ds[SK][SR / 4];  // Delta at the sampled rows, K index major
    } a;
    double red[KG][SR][SC];
  } sh;
  __shared__ int sic[SC];
  __shared__ double red2[8][2];
  __shared__ int last;
  const int tid = threadIdx.x, cl = tid & (SC - 1), kg = tid >> 5;
  const int nblk = kpad / SC;
  const int c0 = (int)(((int64_t)cb * nblk) / ncb) * SC;
  if (tid < SC) sic[tid] = (c0 + tid < k) ? icol[c0 + tid] : -1;
  __syncthreads();
  // this thread's load slots: Z float4 f = tid + 256 q -> column f / (SK/4),
  // rows 4 (f % (SK/4)); Delta float4 f -> sampled row f % SR, columns
  // 4 (f / SR) (a warp's stores into the K-major copy then hit 16 banks)
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
      const int f = tid + 256 * q, r = f % SR, m4 = f / SR;
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
      const float v[4] = {zr[q].x, zr[q].y, zr[q].z, zr[q].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t m = m0 + 4 * m4 + u;
        sh.a.Zs[4 * m4 + u][cc] = v[u] - (m == ic ? 1.f : 0.f);  // W = Z - E
      }
    }
    float* ds = reinterpret_cast<float*>(sh.a.Ds);
#pragma unroll
    for (int q = 0; q < DV; ++q) {
      const int f = tid + 256 * q, r = f % SR, m4 = f / SR;
      const float v[4] = {dr[q].x, dr[q].y, dr[q].z, dr[q].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) ds[(4 * m4 + u) * SR + r] = v[u];
    }
  };
  float hi[SR], lo[SR];
#pragma unroll
  for (int r = 0; r < SR; ++r) hi[r] = lo[r] = 0.f;
  if (k0 < k1) load(k0);
  for (int64_t m0 = k0; m0 < k1; m0 += SK) {
    stash(m0);
    __syncthreads();
    if (m0 + SK < k1) load(m0 + SK);  // in flight during this chunk's products
    float acc[SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) acc[r] = 0.f;
#pragma unroll 4
    for (int mm = kg; mm < SK; mm += KG) {
      const float w = sh.a.Zs[mm][cl];
#pragma unroll
      for (int q = 0; q < SR / 4; ++q) {
        const float4 d = sh.a.Ds[mm][q];
        acc[4 * q] = fmaf(d.x, w, acc[4 * q]);
        acc[4 * q + 1] = fmaf(d.y, w, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(d.z, w, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(d.w, w, acc[4 * q + 3]);
      }
    }
#pragma unroll
    for (int r = 0; r < SR; ++r) two_sum_add(hi[r], lo[r], acc[r]);
    __syncthreads();
  }
  // the K-groups' pairs, added in group order, are this K range's partial
#pragma unroll
  for (int r = 0; r < SR; ++r) sh.red[kg][r][cl] = (double)hi[r] + (double)lo[r];
  __syncthreads();
  double* mine = part + ((int64_t)cb * KS + ks) * SR * SC;
  for (int e = tid; e < SR * SC; e += 256) {
    double tot = 0.0;
    for (int g = 0; g < KG; ++g) tot += sh.red[g][e / SC][e % SC];
    mine[e] = tot;
  }
  // the last of the column block's KS CTAs to arrive adds the ranges in order
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&arrived[cb], 1) == KS - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sum = 0.0, cnt = 0.0;
  const double* blk = part + (int64_t)cb * KS * SR * SC;
  for (int e = tid; e < SR * SC; e += 256) {
    const int r = e / SC, cc = e % SC, c = c0 + cc, ic = sic[cc];
    const int j = r * stride + off;
    if (ic < 0 || j >= n || j == ic) continue;  // the unit entry's P is not used by the map
    double tot = 0.0;
    for (int q = 0; q < KS; ++q) tot += __ldcg(blk + (int64_t)q * SR * SC + e);
    const double exact = tot + (double)Drow[(int64_t)j * ld + ic];
    const double dlt = (double)psmp[(int64_t)r * kpad + c] - exact;
    sum += dlt * dlt;
    cnt += 1.0;
  }
  sum = warp_sum(sum);
  cnt = warp_sum(cnt);
  if ((tid & 31) == 0) {
    red2[tid >> 5][0] = sum;
    red2[tid >> 5][1] = cnt;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0, u = 0.0;
    for (int w = 0; w < 8; ++w) {
      t += red2[w][0];
      u += red2[w][1];
    }
    atomicAdd(&st->acc_dp2, t);
    atomicAdd(&st->acc_dpn, u);
    arrived[cb] = 0;  // ready for the next launch
  }
}

}  // namespace

int64_t sample_scratch_bytes() {
  return (int64_t)kMaxBlocks * KS * SR * SC * 8 + (int64_t)kMaxBlocks * 4;
}

void launch_sample_exact(const float* Drow, const float* Z, const int32_t* icol, int n, int k,
                         int kpad, int64_t ld, const float* psmp, int stride, int off,
                         void* scratch, DevState* st, const DynZ& dz, cudaStream_t s) {
  const int blocks = kpad / SC < kMaxBlocks ? kpad / SC : kMaxBlocks;
  double* part = static_cast<double*>(scratch);
  int* arrived = reinterpret_cast<int*>(part + (int64_t)kMaxBlocks * KS * SR * SC);
  launch_pdl(k_sample_exact, dim3((unsigned)(blocks * KS)), dim3(256), 0, s, Drow, Z, icol, n, k,
             kpad, ld, psmp, stride, off, part, arrived, st, dz);
}

}  // namespace ipt
