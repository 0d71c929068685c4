// Batched solve with tensor-core products (precision bf16x3 / bf16): many
// independent dense problems, Alg. 2 (full spectrum, k = n) for each inside
// one CTA, the map of Eq. (dyn) in the product's epilogue, one persistent
// launch for the whole batch (the control logic is that of the FP32 SIMT
// variant in k_batched.cu).
//
// The product P = Delta_{:,c} + Delta W (W = Z - E) runs on tcgen05 MMAs in
// BF16 hi/lo splits (x = hi + lo to ~16 bits; three passes Dh Wl, Dl Wh,
// Dh Wh, or the single pass Dh Wh), FP32 accumulation in TMEM, the E part
// Delta_jc added exactly in FP32.  Both operands sit in global memory already
// split and in the 128-byte swizzled K-major tile layout of the MMAs:
//   - a prologue kernel (k_batched_tc_prep, one CTA per problem, the whole
//     grid streaming at memory speed) writes Delta's tiles, a column-major
//     FP32 copy DT of Delta for the epilogue's E part, and the product-free
//     first evaluation at Z = E: the tiles of W0 = F0 - E and the sums of its
//     stopping test (F0 itself, -Delta_jc / (theta_j - theta_c) off the
//     diagonal, is recomputed from DT where it is needed: in the first
//     product's epilogue, with the same arithmetic);
//   - W's tiles of every later iterate are written by the epilogue that
//     produces it, into the other of two per-CTA tile sets.
// So a 64-deep slice of a 128 x 128 output tile is two contiguous bulk copies
// (cp.async.bulk, 32 KB each for three passes), and the CTA is warp-
// specialised:
//   warp 16  copies slices into a 3-stage shared-memory ring (mbarriers),
//   warp 17  issues the MMAs of each slice (one thread) into one of two
//            128-column TMEM accumulators and commits them,
//   warps 0-15 run the epilogue of the previous tile meanwhile: tcgen05.ld of
//            the accumulator (warp w reads TMEM lanes 32 (w mod 4).. and the
//            column quarter w / 4, 8 columns at a time), the map, the FP32
//            iterate and W's split tiles for the next evaluation.  (Sixteen
//            epilogue warps at 96 registers issue faster than eight at 164:
//            the epilogue sets the pace.)
// Output tiles go column block by column block, each block's diagonal tile
// first (it yields d_c = Delta_cc + (Delta W)_cc for the block).  Every wait
// is bounded; a wait that gives up ends the CTA's work with
// IPT_DEVICE_TIMEOUT after its copies and MMAs in flight have drained.
#include <cuda_bf16.h>

#include <algorithm>

#include "ipt_internal.cuh"
#include "tc.cuh"

namespace ipt {

namespace {

constexpr int kT = 128;             // output tile rows and columns (B-operand rows)
constexpr int kK = 64;              // product depth per slice: one 128-byte BF16 row
constexpr int kTile = kT * kK * 2;  // one BF16 operand tile, 16 KB
constexpr int kPair = 2 * kTile;    // hi tile, then lo tile
constexpr int kStages = 3;
constexpr int kStage = 2 * kPair;   // A pair + B pair
constexpr int kSmem = kStages * kStage + 1024;
constexpr int kEpiWarps = 16;
constexpr int kEpi = kEpiWarps * 32;
constexpr int kCopyWarp = 16, kMmaWarp = 17;
constexpr int kThreads = kEpi + 64;
constexpr int kTPad = kT + 1;       // row stride of the transposing buffer (floats)
constexpr int kU = 16;              // loads in flight per thread in the output copy
constexpr int kPI = 4;              // prologue: K pairs (8 loads) in flight per thread
static_assert(kK * kTPad * 4 <= kStages * kStage, "transposing buffer fits the ring");
// kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both
// K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kT >> 3) << 17) |
                            ((uint32_t)(kT >> 4) << 24);

struct TcArgs {
  const float* M;        // packed row-major problems
  const double* theta;   // packed partitions (null: diag(M))
  const int64_t* m_off;  // element offset of problem p in M and Z
  const int64_t* v_off;  // element offset of problem p in theta and lambda
  const int* nsz;        // n of problem p
  const int* order;      // schedule: problem indices, largest first
  double* lambda;        // packed eigenvalues
  float* Z;              // packed column-major eigenvector blocks
  int* status;           // per problem: ipt_status
  int* iters;            // per problem: evaluations of F
  uint8_t* ws;           // per CTA: ws_bytes (an iterate, W's two tile sets)
  int64_t ws_bytes;
  int64_t sets_off;      // byte offset of W's tile sets in a CTA's workspace
  int64_t set_bytes;     // one set of split tiles for the largest problem
  const int64_t* t_off;  // byte offset of problem p's tile set in prep_a / prep_w
  uint8_t* prep_a;       // per problem: Delta's split tiles
  uint8_t* prep_w;       // per problem: W0's split tiles
  float* prep_dt;        // per problem (at m_off): DT, column-major Delta
  double* prep_sums;     // per problem and 128-row block: ||F0 - E||^2, ||R0||^2 partials
  int* prep_flag;        // per problem and row block: 1 non-finite theta, 2 degenerate gap
  int max_nt;            // row blocks of the largest problem (slots per problem above)
  int* queue;            // next schedule slot (zero at launch)
  int64_t max_n2;
  int count;
  int max_iter, stop;
  double tol, diverge_bound;
  int passes;            // 3: split x3, 1: hi only
};

struct __align__(16) SmemTc {
  // per column c: theta_c as an FP32 pair and d_c = (Delta Z)_cc of the current
  // evaluation, one 16-byte load in the epilogue
  float4 col[kBatchMaxN];   // (th_hi, th_lo, d, 0)
  float ddiag[kBatchMaxN];  // Delta_jj = M_jj - theta_j (formed in FP64 once per problem)
  F2 red[3][32];
  uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
  uint64_t dbar;  // a diagonal tile's d_c written (the four warps holding the diagonal)
  uint32_t tmem;
  uint32_t gc, gm, tm;  // pipeline positions of the copy and MMA threads (kept here, not
                        // in every thread's registers)
  int abort, prob, flag, verdict;
};

// Byte offset of BF16 element (r, k) in a 128 x 64 K-major tile with 128-byte
// swizzle: 8-row atoms of 1024 B, 16-byte chunk index (k / 8) XOR (r mod 8).
__device__ __forceinline__ int sw128(int r, int k) {
  return (r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) << 4) | ((k & 7) << 1));
}

// x as BF16 hi (and lo = rn(x - hi)) at byte `off` of a tile pair.
__device__ __forceinline__ void put_split(uint8_t* pair, int off, float x, bool with_lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  *reinterpret_cast<__nv_bfloat16*>(pair + off) = h;
  if (with_lo)
    *reinterpret_cast<__nv_bfloat16*>(pair + kTile + off) =
        __float2bfloat16_rn(x - __bfloat162float(h));
}

// Two K-adjacent values (x0 at the even K index, byte offset `off`) as packed
// BF16 hi (and lo) pairs; the same roundings as put_split.
__device__ __forceinline__ void put_split2(uint8_t* pair, int off, float x0, float x1,
                                           bool with_lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  *reinterpret_cast<__nv_bfloat162*>(pair + off) = h;
  if (with_lo) {
    const float2 hf = __bfloat1622float2(h);
    *reinterpret_cast<__nv_bfloat162*>(pair + kTile + off) =
        __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  }
}

// 8 consecutive accumulator columns of this thread's TMEM lane (load and
// completion wait in one asm statement).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(mbar::su32(dst)),
      "l"(src), "r"(bytes), "r"(mbar::su32(bar))
      : "memory");
}

// Output tile ti of an evaluation (nt x nt tiles): column block by column
// block, each starting with its diagonal tile.
__device__ __forceinline__ void tile_of(int ti, int nt, int& rb, int& cb) {
  cb = ti / nt;
  rb = (cb + ti % nt) % nt;
}

constexpr int kPT = 256;  // prologue threads per CTA

// Prologue, one CTA per problem and 128-row block rb (problems largest first;
// max_nt slots per problem, the ones past its blocks return at once).  Per
// 128 x 64 block (rb, ks) of Delta: 2 kPI loads in flight per thread, the BF16
// split tile (rb, ks), and the block transposed through shared memory for the
// column-major outputs: DT and W0's tile entries (row c, K index j; F0_jc =
// -Delta_jc / (theta_j - theta_c) off the diagonal, 1 on it).  Stores go as
// packed BF16 pairs of K-adjacent entries.  W0's rows past the blocks' extent
// are zero padding (written by the rb = 0 CTA).  The first evaluation's sums
// are written per row block and added by the solve kernel in block order.
__global__ void __launch_bounds__(kPT, 4) k_batched_tc_prep(TcArgs a) {
  __shared__ float th_hi[kBatchMaxN], th_lo[kBatchMaxN], ddiag[kBatchMaxN];
  __shared__ float tbuf[kK * kTPad];
  __shared__ F2 red[2][32];
  __shared__ int flag;
  const int tid = threadIdx.x;
  const int p = a.order[blockIdx.x / a.max_nt], rb = blockIdx.x % a.max_nt;
  const int n = a.nsz[p];
  const int nt = (n + kT - 1) / kT, nks = (n + kK - 1) / kK;
  if (rb >= nt) return;  // uniform over the CTA
  const bool three = a.passes == 3;
  const float* M = a.M + a.m_off[p];
  const int64_t vo = a.v_off[p];
  uint8_t* A = a.prep_a + a.t_off[p];
  uint8_t* W = a.prep_w + a.t_off[p];
  float* DT = a.prep_dt + a.m_off[p];
  if (tid == 0) flag = 0;
  __syncthreads();
  for (int j = tid; j < n; j += kPT) {
    const double t = a.theta ? a.theta[vo + j] : (double)M[(int64_t)j * n + j];
    if (!isfinite(t)) atomicOr(&flag, 1);
    const float h = (float)t;
    th_hi[j] = h;
    th_lo[j] = (float)(t - (double)h);
    ddiag[j] = (float)((double)M[(int64_t)j * n + j] - t);
  }
  __syncthreads();
  float s_inc = 0.f, s_r = 0.f;
  const int kw = nks * kK;  // W0's K extent
  for (int ks = 0; ks < nks; ++ks) {
    const int blk = rb * nks + ks;
    uint8_t* pair = A + (int64_t)blk * kPair;
    // items (row r, K pair 2q, 2q + 1): a warp covers one row's 64 K values;
    // kPI items' loads in flight per thread before any store
    for (int base = tid; base < kT * (kK / 2); base += kPI * kPT) {
      float v0[kPI], v1[kPI];
#pragma unroll
      for (int u = 0; u < kPI; ++u) {
        const int it = base + u * kPT, j = rb * kT + (it >> 5), m = ks * kK + 2 * (it & 31);
        const float* row = M + (int64_t)j * n;
        v0[u] = (j < n && m < n) ? row[m] : 0.f;
        v1[u] = (j < n && m + 1 < n) ? row[m + 1] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kPI; ++u) {
        const int it = base + u * kPT, r = it >> 5, ml = 2 * (it & 31);
        const int j = rb * kT + r, m = ks * kK + ml;
        put_split2(pair, sw128(r, ml), (j < n && j == m) ? ddiag[j] : v0[u],
                   (j < n && j == m + 1) ? ddiag[j] : v1[u], three);
        tbuf[ml * kTPad + r] = v0[u];
        tbuf[(ml + 1) * kTPad + r] = v1[u];
      }
    }
    __syncthreads();
    // items (column c = m, row pair j, j + 1): DT and W0's entries (c, j), (c,
    // j + 1); a warp covers 64 rows of one column
    for (int it = tid; it < kK * (kT / 2); it += kPT) {
      const int ml = it >> 6, r = 2 * (it & 63), c = ks * kK + ml, j = rb * kT + r;
      if (j >= kw) continue;  // past W0's K extent (and past n)
      float w[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jj = j + h;
        if (c < n && jj < n) {
          const float djc = tbuf[ml * kTPad + r + h];
          if (jj != c) {
            const float gap = gap2f(th_hi[jj], th_lo[jj], th_hi[c], th_lo[c]);
            if (gap == 0.f) atomicOr(&flag, 2);
            const float f = -djc * recip_nr(gap);
            s_inc = fmaf(f, f, s_inc);
            s_r = fmaf(djc, djc, s_r);
            w[h] = f;
          }
          DT[(int64_t)c * n + jj] = djc;
        }
      }
      put_split2(W + (int64_t)((c >> 7) * nks + (j >> 6)) * kPair, sw128(c & 127, j & 63), w[0],
                 w[1], three);
    }
    __syncthreads();
  }
  // W0's rows c in [nks * 64, nt * 128) (all past n): zero
  const int pad_rows = rb == 0 ? nt * kT - kw : 0, kp = kw / 2;
  for (int it = tid; it < pad_rows * kp; it += kPT) {
    const int c = kw + it / kp, j = 2 * (it % kp);
    put_split2(W + (int64_t)((c >> 7) * nks + (j >> 6)) * kPair, sw128(c & 127, j & 63), 0.f, 0.f,
               three);
  }
  const F2 t_inc = block_sum(F2{s_inc, 0.f}, red[0]);
  const F2 t_r = block_sum(F2{s_r, 0.f}, red[1]);
  if (tid == 0) {
    const int64_t slot = (int64_t)p * a.max_nt + rb;
    a.prep_sums[2 * slot] = f2_value(t_inc);
    a.prep_sums[2 * slot + 1] = f2_value(t_r);
    a.prep_flag[slot] = flag;
  }
  // the tiles are read next by bulk copies (async proxy) of the main kernel
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_batched_tc(TcArgs a) {
  __shared__ SmemTc sh;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool three = a.passes == 3;
  const uint32_t slice_bytes = three ? 2 * kPair : 2 * kTile;
  uint8_t* ws = a.ws + (int64_t)blockIdx.x * a.ws_bytes;
  float* const zs = reinterpret_cast<float*>(ws);  // the iterate buffer paired with Zout
  uint8_t* const setB[2] = {ws + a.sets_off, ws + a.sets_off + a.set_bytes};

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar::mbar_init(&sh.full[s], 1);
      mbar::mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar::mbar_init(&sh.acc_full[b], 1);
      mbar::mbar_init(&sh.acc_empty[b], kEpiWarps);
    }
    mbar::mbar_init(&sh.dbar, 4);
    sh.abort = 0;
    sh.gc = sh.gm = sh.tm = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     mbar::su32(&sh.tmem)),
                 "r"(2 * kT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sh.tmem;
  volatile int* abort = &sh.abort;

  // pipeline positions, kept across problems (barrier phases persist)
  uint32_t te = 0;  // epilogue warps: tiles finished
  uint32_t td = 0;  // epilogue warps: diagonal tiles passed
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
    const int nt = (n + kT - 1) / kT, nks = (n + kK - 1) / kK;
    const float* M = a.M + a.m_off[p];
    const int64_t vo = a.v_off[p];
    const uint8_t* setA = a.prep_a + a.t_off[p];
    const float* DT = a.prep_dt + a.m_off[p];
    for (int j = tid; j < n; j += kThreads) {
      const double t = a.theta ? a.theta[vo + j] : (double)M[(int64_t)j * n + j];
      const float h = (float)t;
      sh.col[j].x = h;
      sh.col[j].y = (float)(t - (double)h);
      sh.col[j].w = 0.f;
      sh.ddiag[j] = (float)((double)M[(int64_t)j * n + j] - t);
      sh.col[j].z = sh.ddiag[j];  // d at Z = E
    }
    if (tid == 0) {
      int f = 0;
      for (int b = 0; b < nt; ++b) f |= a.prep_flag[(int64_t)p * a.max_nt + b];
      sh.flag = f;
    }
    __syncthreads();
    // the first product reads F0 (recomputed from DT: zc == nullptr) and the
    // prologue's W0; later ones the previous epilogue's iterate and tiles.
    // Products write their iterate to the caller's Z block and the CTA's
    // buffer in turn (so the returned iterate is often in place already) and
    // W's tiles to the two sets.
    float* const Zout = a.Z + a.m_off[p];
    const float* zc = nullptr;
    const uint8_t* Bc = a.prep_w + a.t_off[p];
    int nxt = 0;  // workspace slot written by the next product
    double r0 = 0.0;
    int status = IPT_MAXITER, it = 0;
    bool stalled = false;
    // ---------------------------------------------------------- evaluations
    for (it = 0; it < a.max_iter; ++it) {
      float s_inc = 0.f, s_z = 0.f, s_r = 0.f;
      float* zn = nxt ? zs : Zout;
      uint8_t* Bn = setB[nxt];
      if (it > 0) {
        const int ntiles = nt * nt;
        if (warp == kCopyWarp) {
          // ---------------------------------------------- copies
          if (lane == 0) {
            uint32_t gc = sh.gc;  // slices issued
            for (int ti = 0; ti < ntiles && !*abort; ++ti) {
              int rb, cb;
              tile_of(ti, nt, rb, cb);
              for (int ks = 0; ks < nks; ++ks, ++gc) {
                const int s = gc % kStages;
                const uint32_t use = gc / kStages;
                if (!mbar::wait_bounded(&sh.empty[s], (use & 1u) ^ 1u, abort)) {
                  *abort = 1;
                  break;
                }
                uint8_t* st = ring + s * kStage;
                const uint8_t* ga = setA + (int64_t)(rb * nks + ks) * kPair;
                const uint8_t* gb = Bc + (int64_t)(cb * nks + ks) * kPair;
                mbar::mbar_expect_tx(&sh.full[s], slice_bytes);
                if (three) {
                  bulk_g2s(st, ga, kPair, &sh.full[s]);
                  bulk_g2s(st + kPair, gb, kPair, &sh.full[s]);
                } else {
                  bulk_g2s(st, ga, kTile, &sh.full[s]);
                  bulk_g2s(st + kPair, gb, kTile, &sh.full[s]);
                }
              }
            }
            sh.gc = gc;
          }
          __syncwarp();
        } else if (warp == kMmaWarp) {
          // ---------------------------------------------- MMAs
          if (lane == 0) {
            uint32_t gm = sh.gm, tm = sh.tm;  // slices consumed, tiles accumulated
            for (int ti = 0; ti < ntiles && !*abort; ++ti, ++tm) {
              const uint32_t b = tm & 1u, use_b = tm >> 1;
              if (!mbar::wait_bounded(&sh.acc_empty[b], (use_b & 1u) ^ 1u, abort)) {
                *abort = 1;
                break;
              }
              tc::tc_fence_after();
              const uint32_t acc = tmem + b * kT;
              bool ok = true;
              for (int ks = 0; ks < nks; ++ks, ++gm) {
                const int s = gm % kStages;
                const uint32_t use = gm / kStages;
                if (!mbar::wait_bounded(&sh.full[s], use & 1u, abort)) {
                  ok = false;
                  break;
                }
                tc::tc_fence_after();
                const uint32_t sa = mbar::su32(ring + s * kStage);
                const uint32_t sb = sa + kPair;
#pragma unroll
                for (int k = 0; k < kK / 16; ++k) {
                  const uint32_t first = (ks == 0 && k == 0) ? 0u : 1u;
                  const uint64_t ah = tc::sw128_desc(sa + k * 32), bh = tc::sw128_desc(sb + k * 32);
                  if (three) {
                    const uint64_t al = tc::sw128_desc(sa + kTile + k * 32);
                    const uint64_t bl = tc::sw128_desc(sb + kTile + k * 32);
                    tc::mma_f16(acc, ah, bl, kIdesc, first);
                    tc::mma_f16(acc, al, bh, kIdesc, 1u);
                    tc::mma_f16(acc, ah, bh, kIdesc, 1u);
                  } else {
                    tc::mma_f16(acc, ah, bh, kIdesc, first);
                  }
                }
                tc::mma_commit(&sh.empty[s]);  // the slice's stage is free once these finish
              }
              if (!ok) {
                *abort = 1;
                break;
              }
              tc::mma_commit(&sh.acc_full[b]);
            }
            sh.gm = gm;
            sh.tm = tm;
          }
          __syncwarp();
        } else {
          // ---------------------------------------------- epilogue
          const int q = warp & 3, cq = warp >> 2;  // TMEM lane quarter, column quarter
          const int row = q * 32 + lane;
          for (int ti = 0; ti < ntiles; ++ti, ++te) {
            int rb, cb;
            tile_of(ti, nt, rb, cb);
            const int r0t = rb * kT, c0 = cb * kT, j = r0t + row;
            const uint32_t b = te & 1u, use_b = te >> 1;
            if (!mbar::wait_bounded(&sh.acc_full[b], use_b & 1u, abort)) {
              *abort = 1;
              break;
            }
            tc::tc_fence_after();
            const uint32_t taddr = tmem + b * kT + ((uint32_t)(q * 32) << 16) + (uint32_t)(cq * 32);
            if (rb == cb) {
              // d_c = Delta_cc + (Delta W)_cc: the diagonal entries of lane
              // quarter q's rows are columns q*32 .. q*32+31: the column quarter
              // of the quarter's warp with cq == q (warp-uniform test)
              if (cq == q) {
                float v0[16], v1[16];
                __syncwarp();
                tc::tmem_ld16(taddr, v0);
                tc::tmem_ld16(taddr + 16u, v1);
                float dv = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  if (i == lane) dv = v0[i];
                  if (i + 16 == lane) dv = v1[i];
                }
                if (j < n) sh.col[j].z = sh.ddiag[j] + dv;
                __syncwarp();
                if (lane == 0) mbar::mbar_arrive(&sh.dbar);
              }
              // the block's d_c from the other warps (a bounded wait: after a
              // wait elsewhere gave up the results are discarded anyway)
              if (!mbar::wait_bounded(&sh.dbar, td & 1u, abort)) *abort = 1;
              ++td;
            }
            const bool wrow = j < nks * kK;  // rows carrying W entries (zeros past n)
            const float hj = j < n ? sh.col[j].x : 0.f, lj = j < n ? sh.col[j].y : 0.f;
            uint8_t* brow = Bn + (int64_t)(cb * nks + (j < nks * kK ? j / kK : 0)) * kPair;
            const int kin = j % kK;
#pragma unroll 1
            for (int cc = 0; cc < 32; cc += 8) {
              float v[8];
              __syncwarp();  // the TMEM load is warp-collective
              tmem_ld8(taddr + (uint32_t)cc, v);
              if (!wrow) continue;
              const int cl0 = cq * 32 + cc;
              float zv[8], dv[8];  // the chunk's loads all in flight before their use
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int c = c0 + cl0 + i;
                const bool in = j < n && c < n;
                zv[i] = in && zc ? zc[(int64_t)c * n + j] : 0.f;
                dv[i] = in && j != c ? DT[(int64_t)c * n + j] : 0.f;
              }
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int cl = cl0 + i, c = c0 + cl;
                float w = 0.f;
                if (j < n && c < n) {
                  const float pjc = dv[i] + v[i];  // P_jc = Delta_jc (exact) + (Delta W)_jc
                  const float4 cc4 = sh.col[c];
                  const float gap = gap2f(hj, lj, cc4.x, cc4.y);
                  // Z = F0 at the first product
                  const float z = zc ? zv[i] : (j == c ? 1.f : -dv[i] * recip_nr(gap));
                  float f, r;
                  map_entry<float>(z, pjc, cc4.z, gap, j == c, f, r);
                  zn[(int64_t)c * n + j] = f;
                  s_inc = fmaf(f - z, f - z, s_inc);
                  s_z = fmaf(z, z, s_z);
                  s_r = fmaf(r, r, s_r);
                  w = j != c ? f : 0.f;
                }
                put_split(brow, sw128(cl, kin), w, three);
              }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar::mbar_arrive(&sh.acc_empty[b]);
          }
        }
      }
      // W's tiles of the new iterate are read next by bulk copies
      asm volatile("fence.proxy.async.global;" ::: "memory");
      const F2 t_inc = block_sum(F2{s_inc, 0.f}, sh.red[0]);
      const F2 t_z = block_sum(F2{s_z, 0.f}, sh.red[1]);
      const F2 t_r = block_sum(F2{s_r, 0.f}, sh.red[2]);
      if (tid == 0) {
        // the first evaluation's sums come from the prologue's row blocks, added
        // in block order (||Z||^2 = n at Z = E)
        double tr = 0.0, ti = 0.0;
        if (it == 0) {
          for (int b = 0; b < nt; ++b) {
            const int64_t slot = (int64_t)p * a.max_nt + b;
            ti += a.prep_sums[2 * slot];
            tr += a.prep_sums[2 * slot + 1];
          }
        } else {
          tr = f2_value(t_r);
          ti = f2_value(t_inc);
        }
        const double tz = it == 0 ? (double)n : f2_value(t_z);
        if (it == 0) r0 = sqrt(tr);
        const double inc = sqrt(ti) / sqrt(tz);
        const double rho = r0 > 0.0 ? sqrt(tr) / r0 : 0.0;
        int v = IPT_MAXITER;  // continue
        if (*abort)
          v = IPT_DEVICE_TIMEOUT;
        else if (sh.flag)
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
        stalled = status == IPT_DEVICE_TIMEOUT;
        break;
      }
      if (it + 1 == a.max_iter) break;  // MAXITER: the returned Z is the last evaluated
      if (it > 0) {
        zc = zn;
        Bc = Bn;
        nxt ^= 1;
      }
    }
    // ---------------------------------------------------------- outputs
    const int evals = status == IPT_MAXITER ? a.max_iter : it + 1;
    const bool is_e = (it == 0);  // the test passed (or failed hard) at Z = E
    const int n2 = n * n;  // both column-major: a flat copy, kU loads in flight
    // (F0: from DT as in the epilogue)
    if (is_e || zc != Zout) {
      const float* src = zc ? zc : DT;
      for (int base = tid; base < n2; base += kU * kThreads) {
        float v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int e = base + u * kThreads;
          v[u] = (e < n2 && !is_e) ? src[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int e = base + u * kThreads, c = e / n, j = e - c * n;
          if (e >= n2) continue;
          float z = j == c ? 1.f : 0.f;
          if (!is_e && zc) {
            z = v[u];
          } else if (!is_e && j != c) {
            z = -v[u] * recip_nr(gap2f(sh.col[j].x, sh.col[j].y, sh.col[c].x, sh.col[c].y));
          }
          Zout[e] = z;
        }
      }
    }
    for (int c = tid; c < n; c += kThreads) {
      const double t = a.theta ? a.theta[vo + c] : (double)M[(int64_t)c * n + c];
      a.lambda[vo + c] = t + (double)sh.col[c].z;
    }
    if (tid == 0) {
      a.status[p] = status;
      a.iters[p] = evals;
    }
    __syncthreads();
    if (stalled) {  // uniform: a wait gave up; take no more problems
      cta_stalled = true;
      break;
    }
  }
  if (cta_stalled) {
    // drain: the last copy and the last MMAs issued complete (bounded waits
    // that ignore the abort flag) before the accumulators are freed
    __shared__ int no_abort;
    if (tid == 0) no_abort = 0;
    __syncthreads();
    if (warp == kCopyWarp && lane == 0 && sh.gc > 0) {
      const uint32_t last = sh.gc - 1;
      mbar::wait_bounded(&sh.full[last % kStages], (last / kStages) & 1u, &no_abort,
                         mbar::kWaitLimitNs / 4);
    }
    if (warp == kMmaWarp && lane == 0 && sh.gm > 0) {
      const uint32_t last = sh.gm - 1;
      mbar::wait_bounded(&sh.empty[last % kStages], (last / kStages) & 1u, &no_abort,
                         mbar::kWaitLimitNs / 4);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kT)
                 : "memory");
}

int64_t round_1k(int64_t b) { return (b + 1023) / 1024 * 1024; }

}  // namespace

int64_t batched_tc_tile_bytes(int64_t n) {
  const int64_t nt = (n + kT - 1) / kT, nks = (n + kK - 1) / kK;
  return nt * nks * kPair;
}

// Per-CTA workspace (1 KB aligned parts): one FP32 iterate (max_n^2 floats)
// and W's two split tile sets.
int64_t batched_tc_workspace(int64_t max_n) {
  return round_1k(max_n * max_n * 4) + 2 * batched_tc_tile_bytes(max_n);
}

// The prologue's outputs for the whole batch (1 KB aligned parts): Delta's
// and W0's split tiles (tiles_total bytes each), DT (total_n2 floats), the
// sums (2 doubles) and the flag of every problem's row blocks.
int64_t batched_tc_prep_bytes(int64_t tiles_total, int64_t total_n2, int count, int64_t max_n) {
  const int64_t slots = (int64_t)count * ((max_n + kT - 1) / kT);
  return 2 * round_1k(tiles_total) + round_1k(total_n2 * 4) + round_1k(slots * 16) +
         round_1k(slots * 4);
}

cudaError_t launch_batched_tc(const float* M, const double* theta, const int64_t* m_off,
                              const int64_t* v_off, const int64_t* t_off, const int* nsz,
                              const int* order, int count, int64_t max_n, int64_t tiles_total,
                              int64_t total_n2, double tol, int max_iter, int stop,
                              double diverge_bound, double* lambda, float* Z, int* status,
                              int* iters, void* ws, void* prep, int* queue, int ctas, int passes,
                              cudaStream_t s) {
  static int configured = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured != dev) {
    e = cudaFuncSetAttribute(k_batched_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  TcArgs a;
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
  a.ws = static_cast<uint8_t*>(ws);
  a.ws_bytes = batched_tc_workspace(max_n);
  a.sets_off = round_1k(max_n * max_n * 4);
  a.set_bytes = batched_tc_tile_bytes(max_n);
  a.t_off = t_off;
  uint8_t* q = static_cast<uint8_t*>(prep);
  a.prep_a = q;
  q += round_1k(tiles_total);
  a.prep_w = q;
  q += round_1k(tiles_total);
  a.prep_dt = reinterpret_cast<float*>(q);
  q += round_1k(total_n2 * 4);
  a.max_nt = (int)((max_n + kT - 1) / kT);
  const int64_t slots = (int64_t)count * a.max_nt;
  a.prep_sums = reinterpret_cast<double*>(q);
  q += round_1k(slots * 16);
  a.prep_flag = reinterpret_cast<int*>(q);
  a.queue = queue;
  a.max_n2 = max_n * max_n;
  a.count = count;
  a.max_iter = max_iter;
  a.stop = stop;
  a.tol = tol;
  a.diverge_bound = diverge_bound;
  a.passes = passes == 3 ? 3 : 1;
  k_batched_tc_prep<<<(unsigned)slots, kPT, 0, s>>>(a);
  k_batched_tc<<<ctas, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ipt
