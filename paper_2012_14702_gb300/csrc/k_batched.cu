// Many independent dense problems in one persistent launch: Alg. 2 (full
// spectrum, k = n) for each problem, with its own stopping test, inside one
// CTA.  CTAs take problems from a queue ordered largest first, iterate the
// map of Eq. (dyn) on them to the end without any host round trip, write
// Lambda, Z, a status and an evaluation count, and take the next problem.
//
// Per evaluation and problem (n <= kBatchMaxN):
//   first evaluation, Z = E: no product; F_jc = -Delta_jc / (theta_j - theta_c)
//     off the diagonal, d_c = Delta_cc, R = the off-diagonal part of Delta
//     (its norm is ||R0||, so rho(E) = 1);
//   later ones: P = Delta_{:,c} + Delta W (W = Z - E, FP32 SIMT product in
//     64 x 64 tiles staged through shared memory, the next stage fetched into
//     registers during the current one) with the map applied in the tile
//     epilogue; each column block's diagonal tile goes first and yields
//     d_c = P_cc for the block.
// The iterate lives row-major in a per-CTA scratch pair (ping-pong); the
// returned Z is transposed into the caller's column-major block.
//
// Tensor-core variant (k_batched<true>, BF16 products): the same loop with
// P = Delta_{:,c} + Delta W from tcgen05 MMAs.  Per 128 x 128 output tile and
// 64-deep slice of the product, the CTA's threads convert the slice of Delta
// and of W to BF16 hi/lo pairs (x = hi + lo to ~16 bits) and store them in
// shared memory in the 128-byte swizzled K-major layout; one thread issues
// the MMAs (3 passes: Dh Wl, Dl Wh, Dh Wh, the corrections first; or 1 pass:
// Dh Wh) into a 128-column TMEM accumulator and commits them to a barrier
// that every thread waits on (bounded).  The epilogue reads the accumulator
// with tcgen05.ld, one TMEM lane (row) per thread, two warps per lane quarter
// splitting the columns.  Here the iterate is kept column-major, so the
// epilogue's loads and stores along a warp's 32 rows are contiguous.
#include <cuda_bf16.h>

#include <algorithm>

#include "ipt_internal.cuh"
#include "tc.cuh"

namespace ipt {

namespace {

constexpr int TB = 64;   // largest output tile (rows and columns)
constexpr int TK = 32;   // product depth per shared-memory stage
constexpr int NT = 256;  // threads per CTA (16 x 16, 4 x 4 outputs each)

struct BatchArgs {
  const float* M;         // packed row-major problems
  const double* theta;    // packed partitions (null: diag(M))
  const int64_t* m_off;   // element offset of problem p in M and Z
  const int64_t* v_off;   // element offset of problem p in theta and lambda
  const int* nsz;         // n of problem p
  const int* order;       // schedule: problem indices, largest first
  double* lambda;         // packed eigenvalues
  float* Z;               // packed column-major eigenvector blocks
  int* status;            // per problem: ipt_status
  int* iters;             // per problem: evaluations of F
  float* scratch;         // per CTA: 2 * max_n2 floats
  int* queue;             // next schedule slot (zero at launch)
  int64_t max_n2;
  int count;
  int max_iter, stop;
  double tol, diverge_bound;
  int tiles[kBatchClasses];  // output tile (32 or 64) per size class
  int tc_passes;             // tensor-core variant: 1 or 3 BF16 passes
};

__device__ __forceinline__ int batch_class(int n) { return n <= 64 ? 0 : (n <= 256 ? 1 : 2); }

struct __align__(16) Shared {
  float As[TB][TK + 1];  // Delta tile, [row][k]
  float Bs[TK][TB + 4];  // W tile, [k][column]
  float th_hi[kBatchMaxN], th_lo[kBatchMaxN];
  float ddiag[kBatchMaxN];  // Delta_jj = M_jj - theta_j (formed in FP64 once per problem)
  float d[kBatchMaxN];      // d_c = (Delta Z)_cc of the current evaluation
  F2 red[3][32];
  int prob, flag, verdict;
};

// One product evaluation of a problem (P = Delta_{:,c} + Delta W, the map in
// the tile epilogue), output tiles TBT x TBT (32 or 64), each of the 16 x 16
// threads owning R x R outputs.
template <int TBT>
__device__ __forceinline__ void product_map(const BatchArgs& a, const float* __restrict__ M,
                                            int n, const float* __restrict__ zc,
                                            float* __restrict__ zn, Shared& sh, float& s_inc,
                                            float& s_z, float& s_r) {
  constexpr int R = TBT / 16;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  (void)a;
  // P = Delta_{:,c} + Delta W tile by tile, the map in the epilogue.  Each
  // column block starts with its diagonal tile, whose P_cc give the d_c
  // (d_c = (Delta Z)_cc, Eq. dyn) that every tile of the block needs.
  const int nt = (n + TBT - 1) / TBT;
  for (int cb = 0; cb < nt; ++cb)
    for (int rb = 0; rb < nt; ++rb) {
      const int c0t = cb * TBT, r0t = ((cb + rb) % nt) * TBT;
      float acc[R][R] = {};
      // the next stage's tiles are fetched into registers while the
      // current one is multiplied (A: Delta rows r0t.., columns k0..,
      // Delta_jj = M_jj - theta_j formed in FP64; B: W rows k0..,
      // columns c0t.., W_cc = Z_cc - 1 = 0)
      float pa[TBT * TK / NT], pb[TBT * TK / NT];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < TBT * TK / NT; ++r) {
          const int e = tid + r * NT;
          const int j = r0t + e / TK, m = k0 + e % TK;
          float v = 0.f;
          if (j < n && m < n) v = j != m ? M[(int64_t)j * n + m] : sh.ddiag[j];
          pa[r] = v;
          const int m2 = k0 + e / TBT, c = c0t + e % TBT;
          pb[r] = (m2 < n && c < n && m2 != c) ? zc[(int64_t)m2 * n + c] : 0.f;
        }
      };
      auto stage = [&]() {
#pragma unroll
        for (int r = 0; r < TBT * TK / NT; ++r) {
          const int e = tid + r * NT;
          sh.As[e / TK][e % TK] = pa[r];
          sh.Bs[e / TBT][e % TBT] = pb[r];
        }
      };
      fetch(0);
      stage();
      __syncthreads();
      for (int k0 = 0; k0 < n; k0 += TK) {
        const bool more = k0 + TK < n;
        if (more) fetch(k0 + TK);
#pragma unroll 8
        for (int kk = 0; kk < TK; ++kk) {
          float av[R], bv[R];
#pragma unroll
          for (int i = 0; i < R; ++i) {
            av[i] = sh.As[ty * R + i][kk];
            bv[i] = sh.Bs[kk][tx * R + i];
          }
#pragma unroll
          for (int i = 0; i < R; ++i)
#pragma unroll
            for (int q = 0; q < R; ++q) acc[i][q] = fmaf(av[i], bv[q], acc[i][q]);
        }
        __syncthreads();
        if (more) {
          stage();
          __syncthreads();
        }
      }
      if (rb == 0) {  // diagonal tile (uniform over the CTA)
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const int c = c0t + tx * R + q;
            if (ty * R + i == tx * R + q && c < n)
              sh.d[c] = sh.ddiag[c] + acc[i][q];
          }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int j = r0t + ty * R + i;
        if (j >= n) continue;
        float zv[R], mv[R];  // the row's loads all in flight before their use
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int c = c0t + tx * R + q;
          zv[q] = c < n ? zc[(int64_t)j * n + c] : 0.f;
          mv[q] = (c < n && j != c) ? M[(int64_t)j * n + c] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int c = c0t + tx * R + q;
          if (c >= n) continue;
          const float z = zv[q];
          // P_jc = Delta_jc (the E part, exact) + (Delta W)_jc
          const float pjc = mv[q] + acc[i][q];
          const float gap = gap2f(sh.th_hi[j], sh.th_lo[j], sh.th_hi[c], sh.th_lo[c]);
          float f, r;
          map_entry<float>(z, pjc, sh.d[c], gap, j == c, f, r);
          zn[(int64_t)j * n + c] = f;
          s_inc = fmaf(f - z, f - z, s_inc);
          s_z = fmaf(z, z, s_z);
          s_r = fmaf(r, r, s_r);
        }
      }
    }
}

// ---------------------------------------------------------------- tensor-core product
constexpr int TC_T = 128;                    // output tile (rows and columns)
constexpr int TC_K = 64;                     // product depth per shared-memory slice
constexpr int TC_TILE_BYTES = TC_T * TC_K * 2;  // one BF16 operand tile: 16 KB
#ifndef IPT_BATCHED_TC_RG
#define IPT_BATCHED_TC_RG 8
#endif
constexpr int TC_RG = IPT_BATCHED_TC_RG;      // rows staged per group (loads in flight)
static_assert(TC_T % (TC_RG * (256 / 32)) == 0, "row groups tile the operand");
constexpr int TC_PAD = TC_T + 1;               // FP32 row stride of the epilogue's Delta tile
constexpr int TC_SMEM = 4 * TC_TILE_BYTES + 2048;  // Dh, Dl, Wh, Wl (+ alignment); the
                                                   // epilogue reuses it for a 128 x 129 FP32 tile
static_assert(TC_T * TC_PAD * 4 <= 4 * TC_TILE_BYTES + 1024, "epilogue tile fits");
// kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both K-major,
// N = 128, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_T >> 3) << 17) |
                              ((uint32_t)(TC_T >> 4) << 24);

struct TcCtx {
  uint8_t* sa_hi;  // 1024-aligned operand tiles in shared memory
  uint8_t* sa_lo;
  uint8_t* sb_hi;
  uint8_t* sb_lo;
  uint64_t* bar;   // MMA completion barrier
  uint32_t tmem;   // accumulator: 128 lanes x 128 columns
  uint32_t phase;  // next completion phase of `bar`
  int* abort;      // shared flag for the bounded waits
};

// Byte offset of 16-byte chunk `ch` (8 BF16 along K) of row `r` in a 128-byte
// swizzled K-major tile: 8-row atoms of 1024 B, chunk index XOR row mod 8.
__device__ __forceinline__ int sw128_offset(int r, int ch) {
  return (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
}

// Two consecutive values as a BF16 hi pair (and lo = x - hi) at byte `off`
// (4-byte aligned) of the hi / lo tiles.
__device__ __forceinline__ void store_split2(float2 x, uint8_t* hi, uint8_t* lo, int off,
                                             bool with_lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = h;
  if (with_lo) {
    const float2 hf = __bfloat1622float2(h);
    *reinterpret_cast<__nv_bfloat162*>(lo + off) = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
  }
}

// One product evaluation of a problem on the tensor cores (column-major
// iterates zc, zn: element (j, c) at c * n + j).  Returns false if a wait
// for the MMAs gave up (the caller stops).
__device__ bool product_map_tc(const BatchArgs& a, const float* __restrict__ M, int n,
                               const float* __restrict__ zc, float* __restrict__ zn,
                               Shared& sh, TcCtx& tcx, float& s_inc, float& s_z, float& s_r) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, ch_half = warp >> 2;      // epilogue: lane quarter, column half
  const bool three = a.tc_passes == 3;
  const uint32_t sah = tc::su32(tcx.sa_hi), sal = tc::su32(tcx.sa_lo);
  const uint32_t sbh = tc::su32(tcx.sb_hi), sbl = tc::su32(tcx.sb_lo);
  const int nt = (n + TC_T - 1) / TC_T;
  for (int cb = 0; cb < nt; ++cb)
    for (int rb = 0; rb < nt; ++rb) {
      // each column block starts with its diagonal tile (it yields d_c)
      const int c0 = cb * TC_T, r0 = ((cb + rb) % nt) * TC_T;
      for (int kc = 0; kc < n; kc += TC_K) {
        // stage: A = Delta rows r0.., B = W^T columns c0.., K = kc..kc+63.  One
        // warp per row (of A and of B, both contiguous along K in memory), lane
        // l taking K = 2l, 2l+1: coalesced loads, one packed BF16 pair per
        // 4-byte store.  Rows go TC_RG at a time, all loads before any store.
#pragma unroll 1
        for (int g = warp; g < TC_T; g += TC_RG * (NT / 32)) {
          float2 va[TC_RG], vb[TC_RG];
          const int m = kc + 2 * lane;
#pragma unroll
          for (int u = 0; u < TC_RG; ++u) {
            const int rr2 = g + u * (NT / 32), j = r0 + rr2, c = c0 + rr2;
            const float* mrow = M + (int64_t)j * n;
            const float* zcol = zc + (int64_t)c * n;
            va[u].x = (j < n && m < n) ? (j != m ? mrow[m] : sh.ddiag[j]) : 0.f;
            va[u].y = (j < n && m + 1 < n) ? (j != m + 1 ? mrow[m + 1] : sh.ddiag[j]) : 0.f;
            vb[u].x = (c < n && m < n && m != c) ? zcol[m] : 0.f;
            vb[u].y = (c < n && m + 1 < n && m + 1 != c) ? zcol[m + 1] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < TC_RG; ++u) {
            const int rr2 = g + u * (NT / 32);
            const int off = sw128_offset(rr2, lane >> 2) + ((lane & 3) << 2);
            store_split2(va[u], tcx.sa_hi, tcx.sa_lo, off, three);
            store_split2(vb[u], tcx.sb_hi, tcx.sb_lo, off, three);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          tc::tc_fence_after();
#pragma unroll
          for (int k = 0; k < TC_K / 16; ++k) {
            const uint32_t first = (kc == 0 && k == 0) ? 0u : 1u;
            const uint64_t ah = tc::sw128_desc(sah + k * 32), bh = tc::sw128_desc(sbh + k * 32);
            if (three) {
              const uint64_t al = tc::sw128_desc(sal + k * 32), bl = tc::sw128_desc(sbl + k * 32);
              tc::mma_f16(tcx.tmem, ah, bl, TC_IDESC, first);
              tc::mma_f16(tcx.tmem, al, bh, TC_IDESC, 1u);
              tc::mma_f16(tcx.tmem, ah, bh, TC_IDESC, 1u);
            } else {
              tc::mma_f16(tcx.tmem, ah, bh, TC_IDESC, first);
            }
          }
          tc::mma_commit(tcx.bar);
        }
        // the slice's MMAs are done (shared memory free, accumulator final
        // after the last slice); the verdict is made uniform over the CTA
        const bool done = mbar::wait_bounded(tcx.bar, tcx.phase, tcx.abort);
        if (!__syncthreads_and(done ? 1 : 0)) return false;
        tcx.phase ^= 1u;
      }
      tc::tc_fence_after();
      const int row = q * 32 + lane, j = r0 + row;
      const uint32_t taddr = tcx.tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch_half * 64);
      if (r0 == c0) {
        // diagonal tile: d_c = Delta_cc + (Delta W)_cc.  The diagonal entries of
        // lane quarter q's rows are columns q*32 .. q*32+31, held by the warp of
        // that quarter whose column half contains them (warp-uniform test).
        const int dcol = q * 32 - ch_half * 64;
        if (dcol >= 0 && dcol < 64) {
          float v0[16], v1[16];
          __syncwarp();
          tc::tmem_ld16(taddr + (uint32_t)dcol, v0);
          tc::tmem_ld16(taddr + (uint32_t)(dcol + 16), v1);
          float dv = 0.f;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i == lane) dv = v0[i];
            if (i + 16 == lane) dv = v1[i];
          }
          if (j < n) sh.d[j] = sh.ddiag[j] + dv;
        }
        __syncthreads();
      }
      // the E part of P for this tile, Delta rows r0.., columns c0.. (off the
      // diagonal), staged in shared memory (free once the MMAs are done) with
      // coalesced loads: the epilogue walks it along a row per thread
      float* sdel = reinterpret_cast<float*>(tcx.sa_hi);
#pragma unroll 1
      for (int g = warp; g < TC_T; g += 2 * (NT / 32)) {  // two rows' loads in flight
        float v[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int jj = r0 + g + u * (NT / 32), c = c0 + t * 32 + lane;
            v[u][t] = (jj < n && c < n && jj != c) ? M[(int64_t)jj * n + c] : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int t = 0; t < 4; ++t) sdel[(g + u * (NT / 32)) * TC_PAD + t * 32 + lane] = v[u][t];
      }
      __syncthreads();
#pragma unroll 1
      for (int cc = 0; cc < 64; cc += 16) {
        float v[16];
        __syncwarp();  // the TMEM load is warp-collective
        tc::tmem_ld16(taddr + (uint32_t)cc, v);
        if (j >= n) continue;
        const float hj = sh.th_hi[j], lj = sh.th_lo[j];
        float zv[16];  // the chunk's iterate loads all in flight before their use
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = c0 + ch_half * 64 + cc + i;
          zv[i] = c < n ? zc[(int64_t)c * n + j] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int cl = ch_half * 64 + cc + i, c = c0 + cl;
          if (c < n) {
            const float z = zv[i];
            // P_jc = Delta_jc (the E part, exact) + (Delta W)_jc
            const float pjc = sdel[row * TC_PAD + cl] + v[i];
            const float gap = gap2f(hj, lj, sh.th_hi[c], sh.th_lo[c]);
            float f, r;
            map_entry<float>(z, pjc, sh.d[c], gap, j == c, f, r);
            zn[(int64_t)c * n + j] = f;
            s_inc = fmaf(f - z, f - z, s_inc);
            s_z = fmaf(z, z, s_z);
            s_r = fmaf(r, r, s_r);
          }
        }
      }
      tc::tc_fence_before();
      __syncthreads();  // the accumulator is read before the next tile's MMAs
    }
  return true;
}

template <bool TC>
__global__ void __launch_bounds__(NT, TC ? 2 : 3)
    k_batched(BatchArgs a) {
  __shared__ Shared sh;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float* z0 = a.scratch + (int64_t)blockIdx.x * 2 * a.max_n2;
  // tensor-core variant: operand tiles, MMA barrier and a TMEM accumulator
  __shared__ uint64_t tc_bar;
  __shared__ uint32_t tc_tmem;
  __shared__ int tc_abort;
  TcCtx tcx{};
  if constexpr (TC) {
    extern __shared__ uint8_t tc_smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    tcx.sa_hi = base;
    tcx.sa_lo = base + TC_TILE_BYTES;
    tcx.sb_hi = base + 2 * TC_TILE_BYTES;
    tcx.sb_lo = base + 3 * TC_TILE_BYTES;
    if (tid == 0) {
      mbar::mbar_init(&tc_bar, 1);
      tc_abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       mbar::su32(&tc_tmem)),
                   "r"(TC_T)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    tcx.bar = &tc_bar;
    tcx.tmem = tc_tmem;
    tcx.phase = 0;
    tcx.abort = &tc_abort;
  }
  bool cta_stalled = false;
  for (;;) {
    if (tid == 0) {
      const int slot = atomicAdd(a.queue, 1);
      sh.prob = slot < a.count ? a.order[slot] : -1;
    }
    __syncthreads();
    const int p = sh.prob;
    __syncthreads();
    if (p < 0) break;
    const int n = a.nsz[p];
    const int tb = a.tiles[batch_class(n)];
    const float* M = a.M + a.m_off[p];
    const int64_t vo = a.v_off[p];
    // theta (given or diag(M)) as an exact FP32 pair; degenerate / non-finite check
    int bad = 0;
    for (int j = tid; j < n; j += NT) {
      const double t = a.theta ? a.theta[vo + j] : (double)M[(int64_t)j * n + j];
      if (!isfinite(t)) bad = 1;
      const float h = (float)t;
      sh.th_hi[j] = h;
      sh.th_lo[j] = (float)(t - (double)h);
      sh.ddiag[j] = (float)((double)M[(int64_t)j * n + j] - t);
    }
    if (tid == 0) sh.flag = 0;
    __syncthreads();
    if (bad) atomicOr(&sh.flag, 1);
    float* zc = z0;
    float* zn = z0 + a.max_n2;
    // element (j, c) of an iterate: row-major (SIMT) or column-major (tensor cores)
    auto at = [&](int j, int c) -> int64_t {
      return TC ? (int64_t)c * n + j : (int64_t)j * n + c;
    };
    double r0 = 0.0;
    int status = IPT_MAXITER, it = 0;
    bool stalled = false;
    // ---------------------------------------------------------- evaluations
    for (it = 0; it < a.max_iter; ++it) {
      // FP32 per-thread sums, CTA sums as FP32 pairs and the test in FP64 on
      // one thread (the FP64 pipe runs at a small fraction of the FP32 rate
      // here, so no per-entry or per-thread FP64 work)
      float s_inc = 0.f, s_z = 0.f, s_r = 0.f;
      if (it == 0) {
        // Z = E: product-free
        for (int j = ty; j < n; j += NT / 16)
          for (int c = tx; c < n; c += 16) {
            const float djc = M[(int64_t)j * n + c];
            float f = 1.f, r = 0.f;
            if (j != c) {
              const float gap = gap2f(sh.th_hi[j], sh.th_lo[j], sh.th_hi[c], sh.th_lo[c]);
              if (gap == 0.f) atomicOr(&sh.flag, 2);
              f = -djc * recip_nr(gap);
              r = djc;
              s_inc = fmaf(f, f, s_inc);
            } else {
              sh.d[c] = sh.ddiag[c];
            }
            s_r = fmaf(r, r, s_r);
            zn[at(j, c)] = f;
          }
        s_z = tid == 0 ? (float)n : 0.f;
      } else if constexpr (TC) {
        if (!product_map_tc(a, M, n, zc, zn, sh, tcx, s_inc, s_z, s_r)) {
          stalled = true;
          status = IPT_DEVICE_TIMEOUT;
          break;
        }
      } else {
        if (tb == 32) product_map<32>(a, M, n, zc, zn, sh, s_inc, s_z, s_r);
        else product_map<64>(a, M, n, zc, zn, sh, s_inc, s_z, s_r);
      }
      // norms of this evaluation, Alg. 2's test, divergence, cap
      const F2 t_inc = block_sum(F2{s_inc, 0.f}, sh.red[0]);
      const F2 t_z = block_sum(F2{s_z, 0.f}, sh.red[1]);
      const F2 t_r = block_sum(F2{s_r, 0.f}, sh.red[2]);
      if (tid == 0) {  // the totals are valid in thread 0
        const double tr = f2_value(t_r), tz = f2_value(t_z);
        if (it == 0) r0 = sqrt(tr);
        const double inc = sqrt(f2_value(t_inc)) / sqrt(tz);
        const double rho = r0 > 0.0 ? sqrt(tr) / r0 : 0.0;
        int v = IPT_MAXITER;  // continue
        if (sh.flag)
          v = IPT_DEGENERATE_THETA;
        else if (!isfinite(inc) || !isfinite(rho) || sqrt(tz) > a.diverge_bound * sqrt((double)n))
          v = IPT_DIVERGED;
        else if ((a.stop == IPT_STOP_INCREMENT ? inc : rho) <= a.tol)
          v = IPT_OK;
        sh.verdict = v;
      }
      __syncthreads();
      if (sh.verdict != IPT_MAXITER) {
        status = sh.verdict;
        break;
      }
      if (it + 1 == a.max_iter) break;  // MAXITER: the returned Z is the last evaluated
      float* t = zc;
      zc = zn;
      zn = t;
    }
    // ---------------------------------------------------------- outputs
    const int evals = status == IPT_MAXITER ? a.max_iter : it + 1;
    // the returned iterate: E if the test passed (or failed hard) at the first evaluation
    const bool is_e = (it == 0);
    float* Zout = a.Z + a.m_off[p];
    for (int c = ty; c < n; c += NT / 16)
      for (int j = tx; j < n; j += 16)
        Zout[(int64_t)c * n + j] = is_e ? (j == c ? 1.f : 0.f) : zc[at(j, c)];
    for (int c = tid; c < n; c += NT) {
      const double t = a.theta ? a.theta[vo + c] : (double)M[(int64_t)c * n + c];
      a.lambda[vo + c] = t + (double)sh.d[c];
    }
    if (tid == 0) {
      a.status[p] = status;
      a.iters[p] = evals;
    }
    __syncthreads();
    if (stalled) {  // uniform: the MMA wait gave up; take no more problems
      cta_stalled = true;
      break;
    }
  }
  if constexpr (TC) {
    // after a wait that gave up, give the MMAs in flight one more bounded wait
    // before the accumulator is freed
    if (cta_stalled && tid == 0) mbar::wait_bounded(tcx.bar, tcx.phase, tcx.abort);
    tc::tc_fence_before();
    __syncthreads();
    if ((tid >> 5) == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tcx.tmem),
                   "r"(TC_T)
                   : "memory");
  }
}

cudaError_t configure_tc() {
  static int configured = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(k_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e == cudaSuccess) configured = dev;
  return e;
}

}  // namespace

cudaError_t launch_batched(const float* M, const double* theta, const int64_t* m_off,
                           const int64_t* v_off, const int* nsz, const int* order, int count,
                           int64_t max_n2, double tol, int max_iter, int stop,
                           double diverge_bound, double* lambda, float* Z, int* status,
                           int* iters, float* scratch, int* queue, const int* tiles, int ctas,
                           int tc_passes, cudaStream_t s) {
  BatchArgs a;
  a.tc_passes = tc_passes;
  for (int c = 0; c < kBatchClasses; ++c) a.tiles[c] = tiles[c] == 32 ? 32 : 64;
  a.M = M;
  a.theta = theta;
  a.m_off = m_off;
  a.v_off = v_off;
  a.nsz = nsz;
  a.order = order;
  a.lambda = lambda;
  a.Z = Z;
  a.status = status;
  a.iters = iters;
  a.scratch = scratch;
  a.queue = queue;
  a.max_n2 = max_n2;
  a.count = count;
  a.max_iter = max_iter;
  a.stop = stop;
  a.tol = tol;
  a.diverge_bound = diverge_bound;
  if (tc_passes) {
    const cudaError_t e = configure_tc();
    if (e != cudaSuccess) return e;
    k_batched<true><<<ctas, NT, TC_SMEM, s>>>(a);
  } else {
    k_batched<false><<<ctas, NT, 0, s>>>(a);
  }
  return cudaGetLastError();
}

int batched_ctas_per_sm(int tc) {
  int nb = 0;
  if (!tc) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<false>, NT, 0) !=
            cudaSuccess ||
        nb < 1)
      nb = 1;
    return nb;
  }
  // tensor-core variant: from its shared memory and registers per CTA (each
  // resident CTA also holds a 128-column TMEM accumulator: at most four per SM)
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  cudaFuncAttributes fa{};
  if (configure_tc() != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_batched<true>) != cudaSuccess)
    return 1;
  const int per_cta_smem = (int)fa.sharedSizeBytes + TC_SMEM + reserved;
  const int regs = ((fa.numRegs + 7) / 8) * 8 * NT;
  nb = smem_sm / per_cta_smem;
  if (regs > 0) nb = std::min(nb, regs_sm / regs);
  nb = std::min(nb, 4);
  return nb < 1 ? 1 : nb;
}

}  // namespace ipt
