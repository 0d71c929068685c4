// One IPT evaluation on CUDA cores, and the device-side controller.
//
//  k_prepass     d_c = (Delta Z)_{cols[c], c}: the diagonal D(Delta Z) of
//                Eq. (dyn), computed before the product so that every tile of
//                the product can apply the map in its epilogue.
//  k_prepass_tc  the same, plus the tensor-core B operand: W = Z - E scaled by
//                a power of two per column and split into 16-bit hi + lo.
//  k_gemm_simt   P = Delta Z (FP64 or FP32 FMA) with the fused epilogue
//                F = E + G o (Z D(Delta Z) - P) and the norm partials of the
//                stopping test (Alg. 2) and of the residual.
//  k_residual    ||M Z - Z Lambda||_F in FP64 (verification of a result).
//  k_control     the loop test of Alg. 2 on the device.
#include "ipt_internal.cuh"

#include <math.h>

namespace ipt {

namespace {

// ---------------------------------------------------------------- d = D(Delta Z)
// One warp per column c: the contiguous row cols[c] of row-major Delta dotted
// with the contiguous column c of Z.  FP32 data: compensated FP32 sums per
// lane, FP32 pairs (~44 bits) across lanes; FP64 data: FP64 throughout.
template <typename T>
__global__ void k_prepass(const T* __restrict__ Drow, const T* __restrict__ Z, int64_t ld,
                          const int32_t* __restrict__ icol, int kpad, double* __restrict__ d,
                          const DevState* st) {
  if (st->done) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= kpad) return;
  int c = warp, i = icol[c];
  if (i < 0) {
    if (lane == 0) d[c] = 0.0;
    return;
  }
  const T* a = Drow + (int64_t)i * ld;
  const T* z = Z + (int64_t)c * ld;
  double tot;
  if constexpr (sizeof(T) == 4) {
    float s = 0.f, comp = 0.f;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    for (int64_t m = lane; m < ld / 4; m += 32) {
      float4 x = __ldg(a4 + m), y = __ldg(z4 + m);
      float y0 = x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
      float yy = y0 - comp;
      float t = s + yy;
      comp = (t - s) - yy;
      s = t;
    }
    tot = f2_value(warp_sum(F2{s, -comp}));
  } else {
    double s = 0.0;
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const double2* z2 = reinterpret_cast<const double2*>(z);
    for (int64_t m = lane; m < ld / 2; m += 32) {
      double2 x = a2[m], y = z2[m];
      s += x.x * y.x + x.y * y.y;
    }
    tot = warp_sum(s);
  }
  if (lane == 0) d[c] = tot;
}

// V = Z - Z_base on one float4 of column c: Z_base = E (the unit entry at
// row i) when b4 is null, else the stored base iterate.
__device__ __forceinline__ void subtract_base(float4& y, const float4* b4, int m, int i) {
  if (b4) {
    const float4 b = b4[m];
    y.x -= b.x;
    y.y -= b.y;
    y.z -= b.z;
    y.w -= b.w;
  } else {
    const int off = i - 4 * m;
    y.x -= off == 0 ? 1.f : 0.f;
    y.y -= off == 1 ? 1.f : 0.f;
    y.z -= off == 2 ? 1.f : 0.f;
    y.w -= off == 3 ? 1.f : 0.f;
  }
}

// Device-chosen operands: the W set the product reads (wh / wl [wsel]), and the
// next operand written by the previous product's epilogue (DevState::vb).  With
// it, d_c is the sum of that epilogue's partials over 32-row groups,
// dpart[c * G + g], added in a fixed order (lanes over g, then a butterfly) so
// that it does not depend on the order in which the product's CTAs ran; the
// column scale is the state's.  Called by one whole warp per column c.
__device__ __forceinline__ void prepass_handover(const DevState* st, const DynZ& dz, int c,
                                                 int lane, double* d, float* sinv) {
  const double* p = dz.dpart + (int64_t)c * dz.dgroups;
  double s = 0.0;
  for (int g = lane; g < dz.dgroups; g += 32) s += p[g];
  s = warp_sum(s);
  if (lane == 0) {
    d[c] = s;
    sinv[c] = st->wscale;
  }
}

// One warp per column c: d_c as in k_prepass (compensated FP32 per lane,
// FP32 pairs across lanes) and max |W_.c|; then W_.c * s_c split into hi/lo
// (the column is re-read from cache).  Padding columns only get d = 0.
template <bool BF16>
__global__ void k_prepass_tc(const float* __restrict__ Drow, const float* __restrict__ Z,
                             const float* __restrict__ Zbase, int64_t ld,
                             const int32_t* __restrict__ icol, int kpad,
                             double* __restrict__ d, uint16_t* __restrict__ Wh,
                             uint16_t* __restrict__ Wl, float* __restrict__ sinv,
                             const DevState* st, DynZ dz) {
  griddep_wait();  // launched with programmatic dependent launch
  griddep_launch();
  if (st->done || (dz.dyn && st->pause)) return;
  if (dz.dyn) {
    Z = dz.z[st->cur];
    Zbase = st->base >= 0 ? dz.z[st->base] : nullptr;
    if (dz.wh[0]) {
      Wh = dz.wh[st->wsel & 1];
      Wl = dz.wl[st->wsel & 1];
    }
    if (st->passes != 3) Wl = nullptr;
  }
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= kpad) return;
  if (dz.dyn && dz.dpart && st->split_ready) {  // uniform over the grid
    prepass_handover(st, dz, c, lane, d, sinv);
    return;
  }
  const int i = icol[c];
  if (i < 0) {
    if (lane == 0) {
      d[c] = 0.0;
      sinv[c] = 1.f;
    }
    return;
  }
  const float4* a4 = reinterpret_cast<const float4*>(Drow + (int64_t)i * ld);
  const float4* z4 = reinterpret_cast<const float4*>(Z + (int64_t)c * ld);
  const float4* b4 = Zbase ? reinterpret_cast<const float4*>(Zbase + (int64_t)c * ld) : nullptr;
  float s = 0.f, comp = 0.f, mx = 0.f;
  for (int m = lane; m < ld / 4; m += 32) {
    const float4 x = __ldg(a4 + m);
    float4 y = z4[m];
    const float y0 = x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
    const float yy = y0 - comp;
    const float t = s + yy;
    comp = (t - s) - yy;
    s = t;
    subtract_base(y, b4, m, i);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(y.x), fabsf(y.y)), fmaxf(fabsf(y.z), fabsf(y.w))));
  }
  const double tot = f2_value(warp_sum(F2{s, -comp}));
  mx = warp_max(mx);
  const float sc = pow2_scale(mx);
  uint2* h2 = reinterpret_cast<uint2*>(Wh + (int64_t)c * ld);
  uint2* l2 = reinterpret_cast<uint2*>(Wl + (int64_t)c * ld);
  for (int m = lane; m < ld / 4; m += 32) {
    float4 y = z4[m];
    subtract_base(y, b4, m, i);
    uint16_t h[4], l[4];
    split16(y.x * sc, BF16, h[0], l[0]);
    split16(y.y * sc, BF16, h[1], l[1]);
    split16(y.z * sc, BF16, h[2], l[2]);
    split16(y.w * sc, BF16, h[3], l[3]);
    h2[m] = make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
    if (Wl) l2[m] = make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
  }
  if (lane == 0) {
    d[c] = tot;
    sinv[c] = 1.f / sc;
  }
}

// The same pre-pass with the column held in registers (V = Z - Z_base): a CTA
// per column at a time, on a persistent grid of a few CTAs per SM that walks
// the columns (a launch that only hands over the epilogue's operand, or
// returns at entry, then costs a few microseconds instead of a grid of kpad
// CTAs); each thread owns up to VPT float4 slots of the column, so Z is read
// from memory once (the two-pass warp kernel above re-reads the column, which
// at n = 8192 no longer fits in L1/L2 between its passes).  Used when
// npad <= 4*VPT*1024.
template <bool BF16, int VPT>
__global__ void __launch_bounds__(1024)
    k_prepass_tc_reg(const float* __restrict__ Drow, const float* __restrict__ Z,
                     const float* __restrict__ Zbase, int64_t ld,
                     const int32_t* __restrict__ icol, int kpad, double* __restrict__ d,
                     uint16_t* __restrict__ Wh, uint16_t* __restrict__ Wl,
                     float* __restrict__ sinv, const DevState* st, DynZ dz) {
  griddep_wait();  // launched with programmatic dependent launch
  griddep_launch();
  if (st->done || (dz.dyn && st->pause)) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = blockDim.x >> 5;
  if (dz.dyn) {
    Z = dz.z[st->cur];
    Zbase = st->base >= 0 ? dz.z[st->base] : nullptr;
    if (dz.wh[0]) {
      Wh = dz.wh[st->wsel & 1];
      Wl = dz.wl[st->wsel & 1];
    }
    if (st->passes != 3) Wl = nullptr;
    if (dz.dpart && st->split_ready) {  // uniform over the grid: a warp per column
      for (int c = blockIdx.x * nw + wid; c < kpad; c += gridDim.x * nw)
        prepass_handover(st, dz, c, lane, d, sinv);
      return;
    }
  }
  const int n4 = (int)(ld / 4);
  __shared__ F2 rs[32];
  __shared__ float rm[32];
  for (int c = blockIdx.x; c < kpad; c += gridDim.x) {  // block-uniform
    const int i = icol[c];
    if (i < 0) {
      if (tid == 0) {
        d[c] = 0.0;
        sinv[c] = 1.f;
      }
      continue;
    }
    const float4* a4 = reinterpret_cast<const float4*>(Drow + (int64_t)i * ld);
    const float4* z4 = reinterpret_cast<const float4*>(Z + (int64_t)c * ld);
    const float4* b4 = Zbase ? reinterpret_cast<const float4*>(Zbase + (int64_t)c * ld) : nullptr;
    float4 y[VPT];
    float s = 0.f, comp = 0.f, mx = 0.f;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int m = tid + q * blockDim.x;
      y[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < n4) {
        const float4 x = __ldg(a4 + m);
        y[q] = __ldg(z4 + m);
        const float y0 = x.x * y[q].x + x.y * y[q].y + x.z * y[q].z + x.w * y[q].w;
        const float yy = y0 - comp;
        const float t = s + yy;
        comp = (t - s) - yy;
        s = t;
        subtract_base(y[q], b4, m, i);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(y[q].x), fabsf(y[q].y)),
                             fmaxf(fabsf(y[q].z), fabsf(y[q].w))));
      }
    }
    // d_c: the lanes' compensated sums (s - comp) reduced as FP32 pairs, the
    // warps' pairs by warp 0
    const F2 ws = warp_sum(F2{s, -comp});
    const float wm = warp_max(mx);
    if (lane == 0) {
      rs[wid] = ws;
      rm[wid] = wm;
    }
    __syncthreads();
    float cmax = 0.f;
    for (int w = 0; w < nw; ++w) cmax = fmaxf(cmax, rm[w]);
    F2 tot{0.f, 0.f};
    if (wid == 0) tot = warp_sum(lane < nw ? rs[lane] : F2{0.f, 0.f});
    __syncthreads();  // rs / rm are reused by the next column
    const float sc = pow2_scale(cmax);
    uint2* h2 = reinterpret_cast<uint2*>(Wh + (int64_t)c * ld);
    uint2* l2 = reinterpret_cast<uint2*>(Wl + (int64_t)c * ld);
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int m = tid + q * blockDim.x;
      if (m < n4) {
        uint16_t h[4], l[4];
        split16(y[q].x * sc, BF16, h[0], l[0]);
        split16(y[q].y * sc, BF16, h[1], l[1]);
        split16(y[q].z * sc, BF16, h[2], l[2]);
        split16(y[q].w * sc, BF16, h[3], l[3]);
        h2[m] = make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
        if (Wl) l2[m] = make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
      }
    }
    if (tid == 0) {
      d[c] = f2_value(tot);
      sinv[c] = 1.f / sc;
    }
  }
}

// ---------------------------------------------------------------- SIMT product + map
// Tile BM x BN x BK, 256 threads as 16 (rows) x 16 (cols); each thread owns
// TM x TN outputs in two halves: rows tm*HM + [0, HM) and BM/2 + tm*HM + [0, HM)
// (likewise for columns), so a thread's rows are contiguous in the
// column-major iterate and the epilogue loads/stores vectors along j.
// A = Delta row-major (lda = ld), B = Z column-major (K = rows contiguous).
// FP32 (WFORM): B = W = Z - E (the unit entry is subtracted as the tile is
// loaded) and the epilogue adds the exact column Delta_{., cols[c]} from the
// column-major copy DT, so the FP32 accumulators carry only Delta W; the
// epilogue also sums ||Delta W||^2 (the product's error model) and stores P
// when a.Pout is set (the evaluation becomes a base).
// COMP > 0 (FP32 only): compensated sums.  Each output's FMAs run in a fresh
// FP32 partial for COMP slabs of BK steps (COMP * BK products), and the
// partials are added into an FP32 pair (hi, lo) by Knuth's TwoSum, so the
// rounding error of the whole K-long sum is that of one COMP * BK-long
// sequential sum plus the pair's ~2^-48, instead of a K-long one.
enum { EPI_MAP = 0, EPI_RESIDUAL = 1 };

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using V4 = float4;
};
template <>
struct Vec<double> {
  using V4 = double2;  // 16-byte vector
};

template <typename T, int BM, int BN, int BK, int TM, int TN, int EPI, int COMP = 0>
__global__ void __launch_bounds__(256)
    k_gemm_simt(const T* __restrict__ A, MapArgs<T> a, const double* __restrict__ lam,
                double* __restrict__ racc) {
  static_assert(COMP == 0 || sizeof(T) == 4, "compensated sums are FP32 only");
  constexpr int HM = TM / 2, HN = TN / 2;
  constexpr int VEC = 16 / sizeof(T);          // elements per 16-byte load
  constexpr int LPR = BK / VEC;                // loads per tile row
  static_assert(BM * BK == 256 * VEC && BN * BK == 256 * VEC, "one vector load per thread");
  using V = typename Vec<T>::V4;
  constexpr bool WFORM = (EPI == EPI_MAP) && sizeof(T) == 4;
  if constexpr (EPI == EPI_MAP) {
    if (a.st->done) return;
  }
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];
  const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
  const int m0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const int64_t ld = a.ld;
  const int K = (int)ld;
  const int lr = tid / LPR, lk = (tid % LPR) * VEC;  // this thread's load slot
  const T* Ap = A + (int64_t)(m0 + lr) * ld + lk;
  const T* Bp = a.Zin + (int64_t)(c0 + lr) * ld + lk;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  // compensated sums: the pair (chi, clo) of each output (COMP > 0)
  constexpr int CM = COMP ? TM : 1, CN = COMP ? TN : 1;
  float chi[CM][CN], clo[CM][CN];
#pragma unroll
  for (int i = 0; i < CM; ++i)
#pragma unroll
    for (int j = 0; j < CN; ++j) chi[i][j] = clo[i][j] = 0.f;

  // column this thread loads, and the row of its unit entry (W-form)
  const int ic_load = WFORM ? a.icol[c0 + lr] : -1;
  V ra = *reinterpret_cast<const V*>(Ap), rb = *reinterpret_cast<const V*>(Bp);
  auto unit = [&](int k0) {
    if constexpr (WFORM) {
      const int off = ic_load - (k0 + lk);
      float4& v = reinterpret_cast<float4&>(rb);
      v.x -= off == 0 ? 1.f : 0.f;
      v.y -= off == 1 ? 1.f : 0.f;
      v.z -= off == 2 ? 1.f : 0.f;
      v.w -= off == 3 ? 1.f : 0.f;
    }
  };
  unit(0);
  auto stash = [&](int buf) {
    const T* pa = reinterpret_cast<const T*>(&ra);
    const T* pb = reinterpret_cast<const T*>(&rb);
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      As[buf][lk + q][lr] = pa[q];
      Bs[buf][lk + q][lr] = pb[q];
    }
  };
  stash(0);
  __syncthreads();
  const int KT = K / BK;
  for (int kt = 0; kt < KT; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < KT) {
      ra = *reinterpret_cast<const V*>(Ap + (kt + 1) * BK);
      rb = *reinterpret_cast<const V*>(Bp + (kt + 1) * BK);
      unit((kt + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < HM; ++i) {
        av[i] = As[buf][kk][tm * HM + i];
        av[HM + i] = As[buf][kk][BM / 2 + tm * HM + i];
      }
#pragma unroll
      for (int j = 0; j < HN; ++j) {
        bv[j] = Bs[buf][kk][tn * HN + j];
        bv[HN + j] = Bs[buf][kk][BN / 2 + tn * HN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    if constexpr (COMP > 0) {
      if ((kt + 1) % COMP == 0 || kt + 1 == KT) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const float x = (float)acc[i][j], h0 = chi[i][j];
            const float sm = __fadd_rn(h0, x);
            const float bv = __fsub_rn(sm, h0);
            const float er = __fadd_rn(__fsub_rn(h0, __fsub_rn(sm, bv)), __fsub_rn(x, bv));
            chi[i][j] = sm;
            clo[i][j] = __fadd_rn(clo[i][j], er);
            acc[i][j] = T(0);
          }
      }
    }
    if (kt + 1 < KT) stash(buf ^ 1);
    __syncthreads();
  }

  // ---------------- fused epilogue
  T s_inc = T(0), s_z = T(0), s_r = T(0), s_pv = T(0);
#pragma unroll
  for (int jj = 0; jj < TN; ++jj) {
    const int c = c0 + (jj < HN ? tn * HN + jj : BN / 2 + tn * HN + (jj - HN));
    if (c >= a.k) continue;
    int ic = -1;
    T dc = T(0), lamc = T(0);
    if constexpr (EPI == EPI_MAP) {
      ic = a.icol[c];
      dc = (T)a.d[c];
    } else {
      lamc = (T)lam[c];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int jb = m0 + (h == 0 ? tm * HM : BM / 2 + tm * HM);
      const int64_t o = (int64_t)c * ld + jb;
      T z[HM], f[HM], dcol[HM];
      *reinterpret_cast<V*>(z) = *reinterpret_cast<const V*>(a.Zin + o);
      if constexpr (WFORM) {
        *reinterpret_cast<V*>(dcol) =
            *reinterpret_cast<const V*>(a.DT + (int64_t)ic * ld + jb);
      }
      if constexpr (HM * sizeof(T) == 32) {
        *reinterpret_cast<V*>(z + VEC) = *reinterpret_cast<const V*>(a.Zin + o + VEC);
      }
#pragma unroll
      for (int q = 0; q < HM; ++q) {
        const int j = jb + q;
        T p;
        if constexpr (COMP > 0) p = __fadd_rn(chi[h * HM + q][jj], clo[h * HM + q][jj]);
        else p = acc[h * HM + q][jj];
        if constexpr (WFORM) {
          s_pv += p * p;  // Delta W (zero in padding rows)
          p += dcol[q];
          if (a.Pout && j < a.n) a.Pout[o + q] = p;
        }
        f[q] = z[q];
        if (j >= a.n) continue;
        if constexpr (EPI == EPI_MAP) {
          T gap;
          if constexpr (sizeof(T) == 8) gap = a.theta[j] - a.theta[ic];
          else gap = gap2f(a.th_hi[j], a.th_lo[j], a.th_hi[ic], a.th_lo[ic]);
          T fv, rv;
          if (gap == T(0) && j != ic) flag_degenerate(a.st);
          map_entry<T>(z[q], p, dc, gap, j == ic, fv, rv);
          f[q] = fv;
          s_inc += (fv - z[q]) * (fv - z[q]);
          s_z += z[q] * z[q];
          s_r += rv * rv;
        } else {
          const T rv = p - z[q] * lamc;  // (M Z)_jc - Z_jc lambda_c
          s_r += rv * rv;
        }
      }
      if constexpr (EPI == EPI_MAP) {
        *reinterpret_cast<V*>(a.Fout + o) = *reinterpret_cast<const V*>(f);
        if constexpr (HM * sizeof(T) == 32) {
          *reinterpret_cast<V*>(a.Fout + o + VEC) = *reinterpret_cast<const V*>(f + VEC);
        }
      }
    }
  }
  // block reduction of the four partial sums
  __shared__ double red[4][8];
  const double b_inc = warp_sum((double)s_inc), b_z = warp_sum((double)s_z),
               b_r = warp_sum((double)s_r), b_pv = warp_sum((double)s_pv);
  const int w = tid >> 5, l = tid & 31;
  if (l == 0) {
    red[0][w] = b_inc;
    red[1][w] = b_z;
    red[2][w] = b_r;
    red[3][w] = b_pv;
  }
  __syncthreads();
  if (w == 0) {
    double x0 = l < 8 ? red[0][l] : 0.0, x1 = l < 8 ? red[1][l] : 0.0,
           x2 = l < 8 ? red[2][l] : 0.0, x3 = l < 8 ? red[3][l] : 0.0;
    x0 = warp_sum(x0);
    x1 = warp_sum(x1);
    x2 = warp_sum(x2);
    x3 = warp_sum(x3);
    if (l == 0) {
      if constexpr (EPI == EPI_MAP) {
        atomicAdd(&a.st->acc_inc2, x0);
        atomicAdd(&a.st->acc_z2, x1);
        atomicAdd(&a.st->acc_r2, x2);
        if constexpr (WFORM) atomicAdd(&a.st->acc_pv2, x3);
      } else {
        atomicAdd(racc, x2);
      }
    }
  }
}

// ---------------------------------------------------------------- first evaluation
// F(E) needs no product: at Z = E, P = Delta E is the column cols[c] of Delta
// (DT, exact), d_c = Delta_{cols[c], cols[c]}, and Eq. (dyn) with Z_jc = 0
// off the unit entry gives F_jc = -Delta_{j, cols[c]} / (theta_j -
// theta_{cols[c]}) and R_jc = Delta_{j, cols[c]}; F = 1, R = 0 at the unit
// entry.  Grid (column c, row block); each thread maps MF_RPT groups of 4
// consecutive rows with 16-byte loads and stores.  A zero gap is collected
// per thread and flagged once per warp.
// Two groups per thread and five CTAs per SM (at most 51 registers): 121 us
// against 162 us for four groups at one CTA per SM's register budget (ncu,
// n = 8192, same box); the kernel is bound by the latency of its loads.
#ifndef IPT_MAPFIRST_RPT
#define IPT_MAPFIRST_RPT 2
#endif
constexpr int MF_RPT = IPT_MAPFIRST_RPT;
#ifndef IPT_MAPFIRST_MINB
#define IPT_MAPFIRST_MINB 5
#endif

__global__ void __launch_bounds__(256, IPT_MAPFIRST_MINB)
    k_map_first(MapArgs<float> a, double* __restrict__ d, float* __restrict__ part) {
  if (a.st->done) return;
  const int c = blockIdx.x;
  const int ic = a.icol[c];
  const int64_t ld = a.ld;
  float s_inc = 0.f, s_z = 0.f, s_r = 0.f;
  bool bad = false;
  if (ic < 0) {
    if (blockIdx.y == 0 && threadIdx.x == 0) d[c] = 0.0;
  } else {
    const float* pc = a.DT + (int64_t)ic * ld;
    const float hi = a.th_hi[ic], li = a.th_lo[ic];
    float4 p4[MF_RPT], h4[MF_RPT], l4[MF_RPT];
#pragma unroll
    for (int q = 0; q < MF_RPT; ++q) {  // all loads first
      const int j0 = ((blockIdx.y * MF_RPT + q) * blockDim.x + threadIdx.x) * 4;
      if (j0 < a.n) {
        p4[q] = *reinterpret_cast<const float4*>(pc + j0);
        h4[q] = *reinterpret_cast<const float4*>(a.th_hi + j0);
        l4[q] = *reinterpret_cast<const float4*>(a.th_lo + j0);
      }
    }
#pragma unroll
    for (int q = 0; q < MF_RPT; ++q) {
      const int j0 = ((blockIdx.y * MF_RPT + q) * blockDim.x + threadIdx.x) * 4;
      if (j0 >= a.n) continue;
      const float pp[4] = {p4[q].x, p4[q].y, p4[q].z, p4[q].w};
      const float hh[4] = {h4[q].x, h4[q].y, h4[q].z, h4[q].w};
      const float ll[4] = {l4[q].x, l4[q].y, l4[q].z, l4[q].w};
      float f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u;
        if (j >= a.n) {
          f[u] = 0.f;  // padding rows stay zero
        } else if (j == ic) {
          f[u] = 1.f;
          s_z += 1.f;
          d[c] = (double)pp[u];
        } else {
          const float gap = gap2f(hh[u], ll[u], hi, li);
          bad |= gap == 0.f;
          f[u] = -pp[u] * recip_nr(gap);
          s_inc = fmaf(f[u], f[u], s_inc);
          s_r = fmaf(pp[u], pp[u], s_r);
        }
      }
      *reinterpret_cast<float4*>(a.Fout + (int64_t)c * ld + j0) =
          make_float4(f[0], f[1], f[2], f[3]);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag_degenerate(a.st);
  // block partials of the three norms (summed by k_sum_norms)
  __shared__ float red[3][8];
  const float w0 = warp_sum(s_inc), w1 = warp_sum(s_z), w2 = warp_sum(s_r);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = w0;
    red[1][w] = w1;
    red[2][w] = w2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {  // three arrays of per-block FP32 partials, one per norm
    float t = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[threadIdx.x][q];
    const int64_t nb = (int64_t)gridDim.x * gridDim.y;
    part[threadIdx.x * nb + (int64_t)blockIdx.x * gridDim.y + blockIdx.y] = t;
  }
}

// One block: the evaluation's norm accumulators from per-block partials
// (summed as FP32 pairs, in a fixed order).
__global__ void __launch_bounds__(1024)
    k_sum_norms(const float* __restrict__ part, int64_t count, DevState* st) {
  __shared__ F2 sh[3][32];
  F2 t0{0.f, 0.f}, t1{0.f, 0.f}, t2{0.f, 0.f};
#pragma unroll 4
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {  // coalesced, loads in flight
    t0 = f2_add(t0, F2{part[i], 0.f});
    t1 = f2_add(t1, F2{part[count + i], 0.f});
    t2 = f2_add(t2, F2{part[2 * count + i], 0.f});
  }
  t0 = block_sum(t0, sh[0]);
  t1 = block_sum(t1, sh[1]);
  t2 = block_sum(t2, sh[2]);
  if (threadIdx.x == 0) {
    st->acc_inc2 += f2_value(t0);
    st->acc_z2 += f2_value(t1);
    st->acc_r2 += f2_value(t2);
  }
}

// ---------------------------------------------------------------- controller
// One thread.  Reads the accumulators of the evaluation that just finished
// (at iterate Z = buffer `cur`), applies the test of Alg. 2, the divergence
// and iteration caps, records history, chooses the next evaluation and
// clears the accumulators.
//
// Error model.  Every product is P = P_b + Delta V with V = Z - Z_b for a base
// (Z_b, P_b): Z_b = E with P_b = Delta E exactly (FP32 SIMT forms and the first
// tensor-core evaluations), or an earlier iterate whose P was stored.  The
// product of V errs by about u * ||Delta V|| (u per product kind, measured
// ||Delta V|| of this evaluation), the stored P_b by its own error e_base, and
// the FP32 map arithmetic by about e_arith * (||R0|| + ||Delta (Z - E)||).  The
// device residual rho therefore differs from the true one by at most about
// e_rel = (e_base + u ||Delta V|| + arithmetic) / ||R0||.  With the guard
// (residual stop), an evaluation stops the solve only if rho + e_rel <= tol.
// A fixed-precision solve whose test holds but whose guard does not ends with
// IPT_INACCURATE; a staged solve goes on and escalates its products.
//
// Staged schedule.  After an evaluation the controller predicts ||Delta V|| of
// the next one as kappa * (bound on ||V||) and uses the 1-pass product when its
// error is below stage_switch (0.1) times the predicted next residual, or below
// tol / 10; otherwise a split product that stores its P as the new base (the
// base error grows by that product's error).  The base error is a floor under
// the residual: when it would leave less than half of tol, the schedule
// re-bases on a compensated FP32 product of Delta (Z - E) instead (base E).
__device__ __forceinline__ bool split_stage(int stage) {
  return stage == IPT_PREC_BF16X3 || stage == IPT_PREC_FP16X3;
}

__device__ void control_step(DevState* st, const ControlArgs& a) {
  if (st->done || st->pause) return;
  st->write_out = 0;  // set again below for the next evaluation
  const int it = st->iter;
  const double z2 = st->acc_z2;
  const double inc = sqrt(st->acc_inc2) / sqrt(z2);
  const double r0 = sqrt(st->r0acc);
  const double rho = r0 > 0.0 ? sqrt(st->acc_r2) / r0 : 0.0;
  const double pv = sqrt(st->acc_pv2);
  const bool host_driven = a.host_base >= -1;
  const int stage = host_driven && a.host_stage >= 0 ? a.host_stage : st->stage;
  const int passes = host_driven && a.host_passes >= 0 ? a.host_passes : st->passes;
  const bool measured = (a.host_measure >= 0 ? a.host_measure : st->measure) != 0;
  if (it < IPT_MAX_HISTORY) {
    st->hist_inc[it] = inc;
    st->hist_rho[it] = rho;
    st->hist_stage[it] = passes == 0 ? -1 : stage;
  }
  if (a.csr_n > 0) st->rows_eval += st->win_hi - st->win_lo;
  if (st->split_ready) st->epi_used++;
  if (passes == 1 && (stage == IPT_PREC_BF16 || stage == IPT_PREC_FP16)) st->stage_iters[0]++;
  else if (passes != 0) st->stage_iters[1]++;
  // this evaluation's predicted error (see above)
  const bool w_form = passes == 0 || stage == IPT_PREC_F32 || stage == IPT_PREC_F32C ||
                      stage == IPT_PREC_F64;  // products relative to E
  const int ebase = a.host_base >= -1 ? a.host_base : st->base;
  const int erebase = a.host_base >= -1 ? a.host_rebase : st->rebase;
  double u = 0.0;
  if (passes > 0) {
    if (stage == IPT_PREC_F32) u = a.u_f32;
    else if (stage == IPT_PREC_F32C) u = a.u_acc;
    else if (stage == IPT_PREC_F64) u = 0.0;
    else u = (passes == 3 || split_stage(stage)) ? a.u_high : a.u_low;
  }
  const bool on_base = !w_form && ebase >= 0;
  const double e_b = on_base ? st->e_base : 0.0;
  const double pw = on_base ? st->pw_base + pv : pv;  // ~ ||Delta (Z - E)||
  // the product's error: sampled (with a safety factor for the sample's
  // spread), else the model
  double e_prod = e_b + u * pv;
  if (measured && a.smp_rows > 0 && st->acc_dpn > 0.0) {
    const double cnt = st->acc_dpn;
    const double entries = (double)(a.n_rows - 1) * (double)a.k;  // off the unit entries
    e_prod = sqrt(st->acc_dp2 * entries / cnt) * (1.25 + 4.0 / sqrt(cnt));
    st->e_meas = e_prod;
  }
  st->acc_dp2 = 0.0;
  st->acc_dpn = 0.0;
  const double e_abs = e_prod + a.e_arith * (r0 + pw);
  const double e_rel = r0 > 0.0 ? e_abs / r0 : 0.0;
  if (a.test) {  // the reported pair is the last tested iterate
    st->inc = inc;
    st->rho = rho;
    st->e_rel = e_rel;
  }
  st->iter = it + 1;
  st->acc_inc2 = 0.0;
  st->acc_z2 = 0.0;
  st->acc_r2 = 0.0;
  st->acc_pv2 = 0.0;
  const double test = a.stop == IPT_STOP_INCREMENT ? inc : rho;
  const bool staged = a.mode == IPT_PREC_STAGED;
  const bool guarded = a.guard && a.stop == IPT_STOP_RESIDUAL;
  const bool met = a.test && test <= a.tol;
  const bool certified = !guarded || rho + e_rel <= a.tol;
  // a met but uncertified test is final (IPT_INACCURATE) once the residual no
  // longer falls (or, fixed precision, once the error model alone takes half
  // of tol) and no more accurate product is left to escalate to
  const double best = st->rho_best > 0.0 ? st->rho_best : INFINITY;
  if (a.test) {
    st->stall = rho > 0.9 * best ? st->stall + 1 : 0;
    st->rho_best = fmin(best, rho);
  }
  // extrapolations test non-monotone residuals: three in a row without progress
  const bool stalled = st->stall >= (a.acx ? 3 : 1);
  const bool can_escalate = (staged || a.accel_staged) && !st->acc_based;
  const bool give_up = met && !certified && !can_escalate &&
                       (stalled || (!staged && !a.accel_staged && e_rel >= 0.5 * a.tol));
  if (a.accel_staged && a.test) {
    // ask for an accurate re-base once the split products' sampled error is a
    // sizeable part of the residual (or blocks the stop), if it would shrink it
    const double e_acc = (a.u_acc * pw + a.e_arith * (r0 + pw)) / fmax(r0, 1e-300);
    st->want_acc = measured && (e_rel >= 0.1 * fmax(rho, a.tol) || (met && !certified)) &&
                   e_acc < 0.5 * e_rel;
  }
  if (erebase && passes > 0) {
    // this evaluation's P is the new base product
    st->e_base = e_prod;
    st->pw_base = pw;
    st->acc_based = stage == IPT_PREC_F32C;
  }
  if (!isfinite(inc) || !isfinite(rho) || sqrt(z2) > a.diverge_bound * sqrt((double)a.k)) {
    st->status = IPT_DIVERGED;
    st->done = 1;
    st->answer = st->cur;
  } else if (met && certified) {
    st->status = IPT_OK;
    st->done = 1;
    st->answer = st->cur;
  } else if (give_up) {
    // the products' arithmetic cannot certify tol
    st->status = IPT_INACCURATE;
    st->done = 1;
    st->answer = st->cur;
  } else if (it + 1 >= a.max_iter) {
    st->status = IPT_MAXITER;
    st->done = 1;
    st->answer = st->cur;
  } else {
    const int cur = st->cur, base = st->base;
    const int out = zbuf_free(cur, base);  // where this evaluation wrote F
    if (staged) {
      double kappa = st->kappa > 0.0 ? st->kappa : r0 / sqrt((double)a.k);
      if (passes > 0 && !w_form && st->sv > 0.0 && pv > 0.0) kappa = pv / st->sv;
      st->kappa = kappa;
      const double sv_after = st->rebase ? 0.0 : st->sv;  // ||Z_t - Z_b|| bound
      const double sv_next = sv_after + a.step_scale * inc * sqrt(z2);  // ||Z_{t+1} - Z_b||
      if (st->rebase) st->base = cur;
      const double prev = st->prev_rho;
      double q = (it > 0 && prev > 0.0) ? rho / prev : inc;
      q = fmin(fmax(q, 1e-3), 1.0);
      const double need = fmax(a.stage_switch * rho * q, 0.1 * a.tol);
      const double rr = fmax(r0, 1e-300);
      const double dv_next = kappa * sv_next;  // predicted ||Delta V|| of the next product
      const double eb = (st->base >= 0 ? st->e_base : 0.0) / rr;
      const double e_low = a.u_low * dv_next / rr;
      const double e_high = a.u_high * dv_next / rr;
      const double pw_next = (st->base >= 0 ? st->pw_base : 0.0) + dv_next;
      const double e_acc = a.u_acc * pw_next / rr;
      // the base error is a floor, not a disturbance of the iteration: it may
      // stand while it leaves half of tol for the residual and the arithmetic
      const double room = fmax(need, 0.5 * a.tol - a.e_arith * (1.0 + pw_next / rr));
      // escalate on the base error known so far (a re-base's is sampled); the
      // split product's own error is sampled when it re-bases
      const bool low_ok = e_low <= need;
      (void)e_high;
      const bool improves = a.escalate && e_acc < 0.5 * eb;
      if (eb > room && improves) {
        st->stage = IPT_PREC_F32C;
        st->passes = 1;
        st->rebase = 1;
        st->accurate = 1;
        if (a.pause_on_acc) st->pause = 1;
      } else if (low_ok) {
        st->stage = a.low_stage;
        st->passes = 1;
        st->rebase = 0;
        st->accurate = eb + e_low <= 0.5 * a.tol;
      } else {
        st->stage = a.high_stage;
        st->passes = 3;
        st->rebase = 1;
        st->accurate = eb + e_high <= 0.5 * a.tol;
      }
      st->measure = st->passes == 3 && a.smp_rows > 0;
      st->sv = sv_next;
      // scale of the operand after the next one, written by the next epilogue:
      // ||Z_{t+2} - Z_b|| <= (re-base at t+1 ? 0 : ||Z_{t+1} - Z_b||) + ||Z_{t+2} - Z_{t+1}||,
      // the last step predicted by this one (the 16-bit range leaves a factor of 4).
      // None (vb = 0) when the next evaluation is predicted to stop the solve.
      const bool likely_last = st->accurate && rho * q <= 0.5 * a.tol;
      st->vb = likely_last ? 0.0 : (st->rebase ? 0.0 : sv_next) + inc * sqrt(z2);
      // the pass count of the evaluation after the next one, predicted the same
      // way one contraction step further: the next epilogue writes the lo part
      // of the operand it forms only for a split product
      const double sv2 = (st->rebase ? 0.0 : sv_next) + a.step_scale * inc * q * sqrt(z2);
      const double need2 = fmax(a.stage_switch * rho * q * q, 0.1 * a.tol);
      st->write_lo = !(a.u_low * kappa * sv2 / rr <= need2);
      // the next evaluation forms the returned iterate when the test after it
      // passes (and its own does not): it also stores F into the caller's Z
      st->write_out = a.out_pred && a.test && !(rho * q <= a.tol) && rho * q * q <= a.tol;
      // slow contraction: hand the solve over to the requested acceleration
      if (a.slow_ratio > 0.0 && a.test && it >= 2 && prev > 0.0 && rho > a.slow_ratio * prev)
        st->pause = 2;
    } else {
      if (passes == 0)  // non-staged solve after its product-free first evaluation
        st->passes = split_stage(stage) ? 3 : 1;
      // sample the product error of an evaluation that may be the last one
      const double prev = st->prev_rho;
      const double q = (it > 0 && prev > 0.0) ? fmin(rho / prev, 1.0) : 1.0;
      st->measure = a.smp_rows > 0 && a.measure_below > 0.0 && rho * q <= a.measure_below;
    }
    if (a.csr_n > 0) {
      // CSR: the next iterate is this evaluation's F; its nonzero rows widened
      // by the band bound the rows where the next F can be nonzero (the window
      // only grows, so rows outside it were never written and are still zero)
      st->z_lo = st->nz_lo;
      st->z_hi = st->nz_hi;
      if (a.csr_window && st->z_hi >= st->z_lo) {
        st->win_lo = min(st->win_lo, max(0, st->z_lo - st->band));
        st->win_hi = (int)max((int64_t)st->win_hi,
                              min((int64_t)a.csr_n, (int64_t)st->z_hi + 1 + st->band));
      }
      st->nz_lo = a.csr_n;
      st->nz_hi = -1;
    }
    if (!a.acx) st->cur = out;
    else if (a.next_cur >= 0) st->cur = a.next_cur;
  }
  // the next operand this evaluation's epilogue wrote (split of F - Z_b(next)
  // and d of F): it is the next one when the next evaluation is a tensor-core
  // product of F on the base the epilogue assumed, as the staged Picard step
  // sets them (cur = F; base = this iterate after a re-base, else unchanged)
  const bool fused_ok = st->fused && !st->split_bad && !st->done && !st->pause &&
                        a.mode == IPT_PREC_STAGED && !a.acx && st->stage != IPT_PREC_F32 &&
                        st->stage != IPT_PREC_F32C && (st->passes != 3 || st->fused_lo);
  if (fused_ok) {
    st->wsel ^= 1;
    st->wscale = st->wscale_next;
  }
  st->split_ready = fused_ok ? 1 : 0;
  st->fused = 0;
  st->split_bad = 0;
  st->prev_rho = rho;
}

__global__ void k_control(DevState* st, ControlArgs a) {
  griddep_wait();
  griddep_launch();
  control_step(st, a);
}

}  // namespace

void launch_prepass(const void* Drow, const void* Z, int f64, int64_t ld, const int32_t* icol,
                    int kpad, double* d, DevState* st, cudaStream_t s) {
  unsigned g = (unsigned)((kpad + 7) / 8);
  if (f64)
    k_prepass<double><<<g, 256, 0, s>>>((const double*)Drow, (const double*)Z, ld, icol, kpad, d,
                                        st);
  else
    k_prepass<float><<<g, 256, 0, s>>>((const float*)Drow, (const float*)Z, ld, icol, kpad, d,
                                       st);
}

#ifndef IPT_PREPASS_VPT
#define IPT_PREPASS_VPT 8  // float4 slots of the column per thread
#endif

void launch_prepass_tc(const float* Drow, const float* Z, const float* Zbase, int64_t ld,
                       const int32_t* icol, int kpad, int bf16, double* d, uint16_t* Wh,
                       uint16_t* Wl, float* sinv, DevState* st, cudaStream_t s,
                       const DynZ& dz) {
  constexpr int VPT = IPT_PREPASS_VPT;
  const int64_t n4 = ld / 4;
  if (n4 <= (int64_t)VPT * 1024) {
    int threads = (int)((n4 + VPT - 1) / VPT);
    threads = ((threads + 31) / 32) * 32;
    // persistent: 2048 threads' worth of CTAs per SM at most, none idle
    static int nsm = 0;
    if (nsm <= 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          nsm <= 0)
        nsm = 148;
    }
    const int per_sm = std::max(1, 2048 / threads);
    const int blocks = std::min(kpad, nsm * per_sm);
    if (bf16)
      launch_pdl(k_prepass_tc_reg<true, VPT>, dim3(blocks), dim3(threads), 0, s, Drow, Z, Zbase,
                 ld, icol, kpad, d, Wh, Wl, sinv, (const DevState*)st, dz);
    else
      launch_pdl(k_prepass_tc_reg<false, VPT>, dim3(blocks), dim3(threads), 0, s, Drow, Z,
                 Zbase, ld, icol, kpad, d, Wh, Wl, sinv, (const DevState*)st, dz);
    return;
  }
  unsigned g = (unsigned)((kpad + 7) / 8);
  if (bf16)
    launch_pdl(k_prepass_tc<true>, dim3(g), dim3(256), 0, s, Drow, Z, Zbase, ld, icol, kpad, d,
               Wh, Wl, sinv, (const DevState*)st, dz);
  else
    launch_pdl(k_prepass_tc<false>, dim3(g), dim3(256), 0, s, Drow, Z, Zbase, ld, icol, kpad, d,
               Wh, Wl, sinv, (const DevState*)st, dz);
}

void launch_gemm_simt_f64(const double* Drow, const MapArgs<double>& a, int npad, int kpad,
                          cudaStream_t s) {
  dim3 g(kpad / 64, npad / 64);
  k_gemm_simt<double, 64, 64, 8, 4, 4, EPI_MAP><<<g, 256, 0, s>>>(Drow, a, nullptr, nullptr);
}

#ifndef IPT_COMP_SLABS
#define IPT_COMP_SLABS 4  // BK-slabs per compensated add: 32 products per FP32 partial
#endif

void launch_gemm_simt_f32(const float* Drow, const MapArgs<float>& a, int npad, int kpad,
                          int compensated, cudaStream_t s) {
  dim3 g(kpad / 128, npad / 128);
  if (compensated)
    k_gemm_simt<float, 128, 128, 8, 8, 8, EPI_MAP, IPT_COMP_SLABS><<<g, 256, 0, s>>>(
        Drow, a, nullptr, nullptr);
  else
    k_gemm_simt<float, 128, 128, 8, 8, 8, EPI_MAP><<<g, 256, 0, s>>>(Drow, a, nullptr,
                                                                      nullptr);
}

void launch_residual_f64(const double* M64, const double* Z64, int64_t ld, const double* lam,
                         int n, int k, int npad, int kpad, double* acc, cudaStream_t s) {
  MapArgs<double> a{};
  a.Zin = Z64;
  a.ld = ld;
  a.n = n;
  a.k = k;
  dim3 g(kpad / 64, npad / 64);
  k_gemm_simt<double, 64, 64, 8, 4, 4, EPI_RESIDUAL><<<g, 256, 0, s>>>(M64, a, lam, acc);
}

void launch_control(DevState* st, ControlArgs a, cudaStream_t s, bool pdl) {
  if (pdl) launch_pdl(k_control, dim3(1), dim3(1), 0, s, st, a);
  else k_control<<<1, 1, 0, s>>>(st, a);
}

void launch_map_first(const MapArgs<float>& a, int npad, int kpad, double* d, double* part,
                      cudaStream_t s) {
  dim3 g(kpad, (npad / 4 + 256 * MF_RPT - 1) / (256 * MF_RPT));
  float* pf = reinterpret_cast<float*>(part);
  k_map_first<<<g, 256, 0, s>>>(a, d, pf);
  k_sum_norms<<<1, 1024, 0, s>>>(pf, (int64_t)g.x * g.y, a.st);
}

}  // namespace ipt
