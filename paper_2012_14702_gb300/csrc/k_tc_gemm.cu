// Tensor-core IPT evaluation for sm_103a: P = Delta Z on tcgen05 with the map
// of Eq. (dyn) applied in the epilogue.
//
// Product.  A base iterate with an accurately known product is split off,
// Z = Z_b + V, so P = P_b + Delta V.  Initially Z_b = E (unit columns) and
// P_b = Delta E is the column cols[c] of Delta, read exactly in FP32; later a
// staged solve re-bases on an iterate whose P it stored.  Only Delta V goes
// through the tensor cores.  Operands are 16-bit (FP16, or BF16)
// hi/lo splits of r_j Delta_j. and s_c W_.c with power-of-two scales r_j, s_c
// (the pre-pass and the setup write them), so
//   passes = 1:  P~ = Dh Wh                      (FP16: ~2^-11 relative)
//   passes = 3:  P~ = Dh Wh + Dh Wl + Dl Wh      (FP16: ~2^-22 relative)
// accumulated in FP32 in TMEM, and Delta V = P~ / (r_j s_c) exactly.  Because
// |V| << 1 near the fixed point, the rounding error is scaled by |V| instead of
// by |Z| ~ 1.  (Dh/Dl/Wh/Wl below hold the splits of Delta and of V.)
//
// Kernel shape: persistent, one CTA per SM, 320 threads.
//   warp 0      TMA producer: 128x64 A tiles and 256x64 B tiles (16-bit,
//               128-byte swizzle) into a 4-stage shared-memory ring
//   warp 1      TMEM allocator and single-thread tcgen05.mma issuer,
//               M=128 N=256 K=16 per instruction, two 256-column
//               accumulators (512 TMEM columns) so the epilogue of tile t
//               overlaps the product of tile t+1
//   warps 2..9  epilogue, two warps per TMEM lane quarter (each owns half of
//               the tile's 256 columns): tcgen05.ld 16 columns at a time, the map
//               F = E + G o (Z D(Delta Z) - P), the residual
//               R = (theta_j - theta_i) Z - (Z d - P), writes F (FP32) and
//               the norm partials of the stopping test.
// Every mbarrier wait is bounded (globaltimer); on expiry the CTA records a
// timeout in DevState, drains its TMA loads and MMAs, frees TMEM and returns.
#include "ipt_internal.cuh"
#include "mbar.cuh"
#include "tc.cuh"

#include <cuda.h>

namespace ipt {

namespace {

using namespace mbar;
using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int A_BYTES = BM * BK * 2;
constexpr int TMEM_COLS = 2 * BN;

// Kernel modes.  SINGLE: one CTA per 128 x 256 tile.  PAIR: 2-CTA clusters
// issuing one paired MMA (cta_group::2, M = 256) per K step; each CTA holds its
// own 128 A rows and one 128-row half of B, so a CTA's shared memory takes
// 32 KB per K step instead of 48 KB for the same 128 x 256 x 64 of its own
// output.  Every operand load is a plain (non-multicast) TMA load.
enum { MODE_SINGLE = 0, MODE_PAIR = 2 };
#ifndef IPT_PAIR_STAGES
#define IPT_PAIR_STAGES 6
#endif
template <int MODE>
struct Shape {
  static constexpr int B_BYTES = (MODE == MODE_PAIR ? BN / 2 : BN) * BK * 2;  // per CTA
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;                       // per CTA
  static constexpr int STAGES = MODE == MODE_PAIR ? IPT_PAIR_STAGES : 4;
};
constexpr int MAX_STAGES = 6;
static_assert(IPT_PAIR_STAGES >= 2 && IPT_PAIR_STAGES <= MAX_STAGES, "pipeline depth");
constexpr int EPI_WARPS = 8;  // two per TMEM lane quarter, each owning half of the columns
constexpr int NUM_THREADS = 64 + 32 * EPI_WARPS;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int EPI_COLS = BN / 2;  // columns of a tile one epilogue warp handles
constexpr uint64_t kTimeoutNs = kWaitLimitNs;
#ifndef IPT_GROUP_M
#define IPT_GROUP_M 8
#endif
constexpr int GROUP_M = IPT_GROUP_M;             // row blocks per L2 raster group

// Order of the three split products in one accumulator.  The two correction
// products (Dh Wl, Dl Wh; ~2^-11 of the total) go first, into a still-small
// accumulator, and the main product Dh Wh last: adding ~1000 tiny partial
// sums into an accumulator that already holds the whole product would round
// each of them against the large value.
#ifndef IPT_SPLIT_INTERLEAVED
#define IPT_SPLIT_INTERLEAVED 0
#endif
#ifndef IPT_CORRECTIONS_FIRST
#define IPT_CORRECTIONS_FIRST 1
#endif

// Per-column data of the current tile, staged by each epilogue warp for the
// columns it owns (one 16-byte load per column instead of five shuffles).
struct __align__(16) ColInfo {
  float d;   // d_c
  float s;   // 1 / s_c (column scale of the W operand)
  float hi;  // theta_{cols[c]} hi / lo
  float lo;
};

struct Ctl {
  ColInfo wcol[EPI_WARPS][EPI_COLS];
  int wic[EPI_WARPS][EPI_COLS];
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
template <int MODE>
constexpr int smem_bytes() {
  return Shape<MODE>::STAGES * Shape<MODE>::STAGE_BYTES + 1024 + (int)sizeof(Ctl) + 64;
}
static_assert(smem_bytes<MODE_PAIR>() <= 227 * 1024, "shared memory");
static_assert(smem_bytes<MODE_SINGLE>() <= 227 * 1024, "shared memory");

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A and B both
// FP16 (0) or both BF16 (1) at bits 7-9 / 10-12, both K-major (bits 15, 16 =
// 0), N >> 3 at bit 17, M >> 4 at bit 24 (M of the whole instruction: 256
// for a CTA pair).
constexpr uint32_t idesc_for(bool bf16, int m) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Shared::cluster address of the object at the same offset as `p` in the CTA
// of cluster rank `rank`.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
  return r;
}
// Arrive (release, cluster scope) on a barrier given by its shared::cluster address.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

// Operand loads carry an L2 policy: with IPT_OPERAND_EVICT_LAST the operand
// panels are marked evict-last, so the epilogue's streamed iterate, P_b and F
// (evict-first) do not push them out of L2 between the tiles that reuse them.
#ifndef IPT_OPERAND_EVICT_LAST
#define IPT_OPERAND_EVICT_LAST 1
#endif
__device__ __forceinline__ uint64_t operand_policy() {
  uint64_t p;
#if IPT_OPERAND_EVICT_LAST
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
#else
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
#endif
  return p;
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                         int y, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

// Load whose completion is counted on an mbarrier of either CTA of the pair
// (`bar` is a shared::cluster address, here always the pair's first CTA).
__device__ __forceinline__ void tma_load_pair(void* dst, const CUtensorMap* map, uint32_t bar,
                                              int x, int y, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Paired MMA (issued by the pair's first CTA): D of each CTA (128 lanes x 256
// columns) += its A rows x both CTAs' B halves.
__device__ __forceinline__ void mma_f16_pair(uint32_t dt, uint64_t ad, uint64_t bd,
                                             uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
// Completion of the pair's MMAs arrives on the barrier at the same offset in
// each CTA of `mask`.
__device__ __forceinline__ void mma_commit_pair_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(su32(bar)),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

__device__ __forceinline__ void tile_coords(int t, int num_m, int num_n, int& mb, int& nb) {
  const int per_group = GROUP_M * num_n;
  const int g = t / per_group;
  const int first = g * GROUP_M;
  const int gm = min(GROUP_M, num_m - first);
  const int r = t - g * per_group;
  mb = first + r % gm;
  nb = r / gm;
}

// Order of the K blocks within one pass: farthest from the tile's own column
// block first, that block last.  Near the fixed point of a near-diagonal
// problem the entries W_mc of a column fall off with |theta_m - theta_c|, so
// the terms with m near the tile's columns dominate each sum.  The tensor
// core's FP32 accumulation loses low bits relative to the running sum at each
// accumulate; adding the many small far terms while the sum is still small and
// the few dominant ones last keeps that loss at a fraction of |P|.
// Sums over the warp's 32 lanes of 8 per-lane values x[0..7] (one per column),
// by recursive halving: at each offset o (16, 8, 4) a lane keeps the half of
// its vector picked by bit o of its index and adds the partner's copy of that
// half; exchanges at offsets 2 and 1 complete the sums.  Lane L returns the
// sum of column (L >> 2).  9 shuffles for 8 sums.
__device__ __forceinline__ float warp_colsum8(float (&x)[8], int lane) {
#pragma unroll
  for (int o = 16, m = 4; o >= 4; o >>= 1, m >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < m; ++i) {
      const float keep = up ? x[i + m] : x[i];
      const float send = up ? x[i] : x[i + m];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float t = x[0] + __shfl_xor_sync(0xffffffffu, x[0], 2);
  return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

#ifndef IPT_K_FAR_FIRST
#define IPT_K_FAR_FIRST 1
#endif
struct KOrder {
  int lo, hi, center;
  __device__ void reset(int nb, int num_kb) {
    lo = 0;
    hi = num_kb - 1;
    center = min((nb * BN + BN / 2) / BK, num_kb - 1);
  }
  __device__ int next() {
#if IPT_K_FAR_FIRST
    return (center - lo >= hi - center) ? lo++ : hi--;
#else
    return lo++;
#endif
  }
};

__device__ __forceinline__ void fail(Ctl* ctl, DevState* st, int code) {
  *reinterpret_cast<volatile int*>(&ctl->abort) = 1;
  atomicCAS(&st->timeout, 0, code);
}

// PAIR (cluster of 2 along M): the same two tiles as one 256 x 256 paired
// product.  Each CTA's producer loads its 128 A rows and its half of B into
// its own shared memory, counting the bytes on the first CTA's full barrier
// (armed by the first CTA for both CTAs' bytes).  Only the first CTA's MMA
// thread issues, and its commits arrive on both CTAs' barriers (stage free,
// accumulator full).  Both CTAs' epilogues read their own TMEM and release
// the accumulator on the first CTA's barrier (16 warp arrivals).
template <int MODE>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmDh, const __grid_constant__ CUtensorMap tmDl,
              const __grid_constant__ CUtensorMap tmWh, const __grid_constant__ CUtensorMap tmWl,
              const __grid_constant__ CUtensorMap tmWh1, const __grid_constant__ CUtensorMap tmWl1,
              MapArgs<float> a, int num_m, int num_n, int num_kb, int passes, uint32_t idesc) {
  constexpr bool CLUSTER = MODE != MODE_SINGLE;
  constexpr bool PAIR = MODE == MODE_PAIR;
  constexpr int STAGES = Shape<MODE>::STAGES;
  constexpr int B_BYTES = Shape<MODE>::B_BYTES;
  constexpr int STAGE_BYTES = Shape<MODE>::STAGE_BYTES;
  griddep_wait();  // launched with programmatic dependent launch (paired mode)
  griddep_launch();
  // uniform over the grid, so over each cluster; a paused solve runs its next
  // evaluation with a kernel of another kind first
  if (a.st->done || (a.dyn && a.st->pause)) return;
  // operands: as launched, or (dyn) chosen by the controller's state
  const float* Zin = a.Zin;
  float* Fout = a.Fout;
  const float* Pbase = a.Pbase;
  int pbase_by_icol = a.pbase_by_icol;
  float* Pout = a.Pout;
  float* psmp = a.psmp;  // sampled P entries (error estimate), or none
  int wset = 0;          // W set the product reads
  // next operand (fused split): its sets, its base (nullptr: E), its scale
  uint16_t* wn_h = nullptr;
  uint16_t* wn_l = nullptr;
  const float* zb_next = nullptr;
  bool zb_is_z = false;  // the next base is this evaluation's iterate (a re-base)
  float sc_next = 1.f;
  if (a.dyn) {
    const int cur = a.st->cur, base = a.st->base;
    passes = a.st->passes;
    Zin = a.zsel[cur];
    Fout = a.zsel[zbuf_free(cur, base)];
    Pbase = base >= 0 ? a.pstore : a.DT;
    pbase_by_icol = base >= 0 ? 0 : 1;
    Pout = a.st->rebase ? a.pstore : nullptr;
    if (!a.st->measure) psmp = nullptr;
    wset = a.st->wsel & 1;
    const double vb = a.st->vb;
    if (a.fuse && vb > 0.0 && vb < 1e30) {
      const int write_lo = a.st->write_lo;  // the lo part only for a split product
      wn_h = a.wnh[wset ^ 1];
      wn_l = write_lo ? a.wnl[wset ^ 1] : nullptr;
      zb_is_z = a.st->rebase != 0;
      zb_next = zb_is_z ? Zin : (base >= 0 ? a.zsel[base] : nullptr);
      sc_next = pow2_scale((float)vb);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->fused = 1;
        a.st->fused_lo = write_lo;
        a.st->wscale_next = 1.f / sc_next;
      }
    }
  }
  // second store of F: the host output, or (device-chosen evaluations) the
  // caller's Z when the state predicts this evaluation forms the result
  float* oz = a.host_f;
  int64_t oz_ld = a.host_ld;
  if (!oz && a.dyn && a.out_z && a.st->write_out) {
    oz = a.out_z;
    oz_ld = a.out_ld;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->out_iter = a.st->iter;
  }
  const CUtensorMap* tmBh = wset ? &tmWh1 : &tmWh;
  const CUtensorMap* tmBl = wset ? &tmWl1 : &tmWl;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + STAGES * STAGE_BYTES);
  volatile int* abort = &ctl->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int rank = CLUSTER ? (int)cluster_rank() : 0;
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->tfull[b], 1);
      mbar_init(&ctl->tempty[b], PAIR ? 2 * EPI_WARPS : EPI_THREADS);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair allocates, collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       su32(&ctl->tmem_base)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       su32(&ctl->tmem_base)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CLUSTER) cluster_sync();  // the peer's barriers are initialised before use
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  // tiles of the schedule: single tiles, or vertical tile pairs per cluster
  const int sched_m = CLUSTER ? num_m / 2 : num_m;
  const int num_tiles = sched_m * num_n;
  const int t_first = CLUSTER ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int t_step = CLUSTER ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  // split products interleaved per K block: a stage is two ring slots holding
  // Dh, Dl, Wh and Wl of one K block, and each K step issues the three MMAs
  // (corrections first), so every operand tile is loaded once instead of in
  // two of the three passes
  const bool inter = IPT_SPLIT_INTERLEAVED && passes == 3;
  const int nstages = inter ? STAGES / 2 : STAGES;
  const int total_kb = inter ? num_kb : passes * num_kb;
  static_assert(STAGES % 2 == 0, "interleaved stages take two slots");

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      const uint64_t pol = operand_policy();
      int pend_parity[STAGES];
      for (int s = 0; s < STAGES; ++s) pend_parity[s] = -1;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = t_first; t < num_tiles && ok; t += t_step) {
        int mb, nb;
        tile_coords(t, sched_m, num_n, mb, nb);
        if (CLUSTER) mb = 2 * mb + rank;
        KOrder ko;
        for (int kb = 0; kb < total_kb; ++kb) {
          if (!wait_bounded(&ctl->empty[stage], phase ^ 1u, abort)) {
            fail(ctl, a.st, 1);
            ok = false;
            break;
          }
          const int pass = kb / num_kb;
          if (kb == pass * num_kb) ko.reset(nb, num_kb);
          const int kx = ko.next() * BK;
          if (inter) {
            uint8_t* a0 = sA + (2 * stage) * A_BYTES;
            uint8_t* b0 = sB + (2 * stage) * B_BYTES;
            if constexpr (PAIR) {
              const uint32_t fb = peer_addr(&ctl->full[stage], 0);
              if (leader) mbar_expect_tx(&ctl->full[stage], 4 * STAGE_BYTES);
              tma_load_pair(a0, &tmDh, fb, kx, mb * BM, pol);
              tma_load_pair(a0 + A_BYTES, &tmDl, fb, kx, mb * BM, pol);
              tma_load_pair(b0, tmBh, fb, kx, nb * BN + rank * (BN / 2), pol);
              tma_load_pair(b0 + B_BYTES, tmBl, fb, kx, nb * BN + rank * (BN / 2), pol);
            } else {
              mbar_expect_tx(&ctl->full[stage], 2 * STAGE_BYTES);
              tma_load(a0, &tmDh, &ctl->full[stage], kx, mb * BM, pol);
              tma_load(a0 + A_BYTES, &tmDl, &ctl->full[stage], kx, mb * BM, pol);
              tma_load(b0, tmBh, &ctl->full[stage], kx, nb * BN, pol);
              tma_load(b0 + B_BYTES, tmBl, &ctl->full[stage], kx, nb * BN, pol);
            }
            pend_parity[stage] = (int)phase;
            if (++stage == nstages) {
              stage = 0;
              phase ^= 1u;
            }
            continue;
          }
          // passes = 1: Dh Wh.  passes = 3: (Dh Wl, Dl Wh, Dh Wh), or with the
          // main product first (Dh Wh, Dh Wl, Dl Wh).
          const int role = passes == 1 ? 0 : (IPT_CORRECTIONS_FIRST ? (pass + 1) % 3 : pass);
          const CUtensorMap* mA = role == 2 ? &tmDl : &tmDh;
          const CUtensorMap* mB = role == 1 ? tmBl : tmBh;
          if constexpr (PAIR) {
            const uint32_t fb = peer_addr(&ctl->full[stage], 0);
            if (leader) mbar_expect_tx(&ctl->full[stage], 2 * STAGE_BYTES);
            tma_load_pair(sA + stage * A_BYTES, mA, fb, kx, mb * BM, pol);
            tma_load_pair(sB + stage * B_BYTES, mB, fb, kx, nb * BN + rank * (BN / 2), pol);
          } else {
            mbar_expect_tx(&ctl->full[stage], STAGE_BYTES);
            tma_load(sA + stage * A_BYTES, mA, &ctl->full[stage], kx, mb * BM, pol);
            tma_load(sB + stage * B_BYTES, mB, &ctl->full[stage], kx, nb * BN, pol);
          }
          pend_parity[stage] = (int)phase;
          if (++stage == nstages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!PAIR || leader) {
        // drain: every issued load lands before the CTA may exit (in a pair
        // the first CTA's full barrier also counts the peer's loads)
        for (int s = 0; s < STAGES; ++s) {
          if (pend_parity[s] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(&ctl->full[s], (uint32_t)pend_parity[s]))
            if (gtimer() - t0 > kTimeoutNs) {
              fail(ctl, a.st, 5);
              break;
            }
        }
      } else if (!ok) {
        // the second CTA of a pair cannot observe its loads (they count on the
        // first CTA's barrier): after an abort give any in flight time to land
        const uint64_t t0 = gtimer();
        while (gtimer() - t0 < 200000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0 && (!PAIR || leader)) {
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool ok = true;
      for (int t = t_first; t < num_tiles && ok; t += t_step) {
        if (!wait_bounded<PAIR>(&ctl->tempty[acc], acc_phase ^ 1u, abort)) {
          fail(ctl, a.st, 2);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(acc * BN);
        for (int kb = 0; kb < total_kb; ++kb) {
          if (!wait_bounded(&ctl->full[stage], phase, abort)) {
            fail(ctl, a.st, 3);
            ok = false;
            break;
          }
          tc_fence_after();
          if (inter) {
            // Dh Wl, Dl Wh, Dh Wh at each K step of the block
            const uint32_t ah = su32(sA + (2 * stage) * A_BYTES), al = ah + A_BYTES;
            const uint32_t bh = su32(sB + (2 * stage) * B_BYTES), bl = bh + B_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint64_t dah = sw128_desc(ah + k * 32), dal = sw128_desc(al + k * 32);
              const uint64_t dbh = sw128_desc(bh + k * 32), dbl = sw128_desc(bl + k * 32);
              if constexpr (PAIR) {
                mma_f16_pair(dt, dah, dbl, idesc, (kb | k) != 0);
                mma_f16_pair(dt, dal, dbh, idesc, true);
                mma_f16_pair(dt, dah, dbh, idesc, true);
              } else {
                mma_f16(dt, dah, dbl, idesc, (kb | k) != 0);
                mma_f16(dt, dal, dbh, idesc, true);
                mma_f16(dt, dah, dbh, idesc, true);
              }
            }
          } else {
            const uint32_t ab = su32(sA + stage * A_BYTES), bb = su32(sB + stage * B_BYTES);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              if constexpr (PAIR)
                mma_f16_pair(dt, sw128_desc(ab + k * 32), sw128_desc(bb + k * 32), idesc,
                             (kb | k) != 0);
              else
                mma_f16(dt, sw128_desc(ab + k * 32), sw128_desc(bb + k * 32), idesc,
                        (kb | k) != 0);
            }
          }
          if constexpr (PAIR) mma_commit_pair_mc(&ctl->empty[stage], (uint16_t)0x3);
          else mma_commit(&ctl->empty[stage]);
          if (++stage == nstages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if constexpr (PAIR) mma_commit_pair_mc(&ctl->tfull[acc], (uint16_t)0x3);
        else mma_commit(&ctl->tfull[acc]);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
      // drain: all issued MMAs complete before TMEM is freed
      if constexpr (PAIR) mma_commit_pair(&ctl->drain);
      else mma_commit(&ctl->drain);
      const uint64_t t0 = gtimer();
      while (!mbar_try(&ctl->drain, 0))
        if (gtimer() - t0 > kTimeoutNs) {
          fail(ctl, a.st, 6);
          break;
        }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2..9)
    const int e = warp - 2;      // epilogue warp index
    const int q = warp & 3;      // TMEM lane quarter this warp may access
    const int h = e >> 2;        // which half of the tile's columns it owns
    const int row = q * 32 + lane;
    const int64_t ld = a.ld;
    ColInfo* wcol = ctl->wcol[e];
    int* wic = ctl->wic[e];
    int acc = 0;
    uint32_t acc_phase = 0;
    float s_inc = 0.f, s_z = 0.f, s_r = 0.f, s_pv = 0.f;
    bool split_bad = false;  // a scaled next-operand entry outside the 16-bit range
    const float split_max = a.fuse_bf16 ? 3.0e38f : 65504.f;
    const uint32_t tempty_pair[2] = {PAIR ? peer_addr(&ctl->tempty[0], 0) : 0u,
                                     PAIR ? peer_addr(&ctl->tempty[1], 0) : 0u};
    for (int t = t_first; t < num_tiles; t += t_step) {
      int mb, nb;
      tile_coords(t, sched_m, num_n, mb, nb);
      if (CLUSTER) mb = 2 * mb + rank;
      const int cbase = nb * BN + h * EPI_COLS;
      // stage this warp's column data (its reads of the previous tile are done)
      __syncwarp();
#pragma unroll
      for (int u = 0; u < EPI_COLS / 32; ++u) {
        const int cc = lane + 32 * u, c = cbase + cc;
        const int ic = a.icol[c];
        ColInfo ci;
        ci.d = (float)a.d[c];
        ci.s = a.sinv[c];
        ci.hi = ic >= 0 ? a.th_hi[ic] : 0.f;
        ci.lo = ic >= 0 ? a.th_lo[ic] : 0.f;
        wcol[cc] = ci;
        wic[cc] = ic;
      }
      __syncwarp();
      if (!wait_bounded(&ctl->tfull[acc], acc_phase, abort)) {
        fail(ctl, a.st, 4);
        break;
      }
      tc_fence_after();
      const int j = mb * BM + row;
      const int grp = (mb * BM + q * 32) >> 5;  // this warp's group of 32 rows
      const bool jok = j < a.n;
      const float hj = a.th_hi[j], lj = a.th_lo[j], rj = a.rinv[j];
      // this row's slot among the sampled rows, or -1
      const int jr = (psmp && j % a.smp_stride == a.smp_off) ? j / a.smp_stride : -1;
      float* prow = jr >= 0 && jr < kSampleRows ? psmp + (int64_t)jr * a.smp_kpad : nullptr;
#pragma unroll 1
      for (int ch = 0; ch < EPI_COLS / 16; ++ch) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) +
                      (uint32_t)(acc * BN + h * EPI_COLS + ch * 16),
                  v);
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {  // two halves of 8 columns (register budget)
          const int c0 = ch * 16 + hf * 8;  // first owned column of this half
          float z[8], pb[8], dl[8], zn[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int ic = wic[c0 + i];
            const bool ok = jok && ic >= 0;
            const int64_t o = (int64_t)(cbase + c0 + i) * ld + j;
            // P_base: column cols[c] of Delta (Z_base = E) or the stored P of column c.
            // Streamed once: evict-first, so the reused operand panels stay in L2.
            const int64_t ob = pbase_by_icol ? (int64_t)ic * ld + j : o;
            z[i] = ok ? __ldcs(Zin + o) : 0.f;
            pb[i] = ok ? __ldcs(Pbase + ob) : 0.f;
            // next operand: Delta_{cols[c], j} (row cols[c] of the row-major Delta)
            // and the next base's entry, when it is neither E nor this iterate
            dl[i] = (wn_h && ok) ? __ldcs(a.drow + (int64_t)ic * ld + j) : 0.f;
            zn[i] = (wn_h && ok && zb_next && !zb_is_z) ? __ldcs(zb_next + o) : 0.f;
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int ic = wic[c0 + i];
            const ColInfo ci = wcol[c0 + i];
            const bool ok = jok && ic >= 0;
            const int64_t o = (int64_t)(cbase + c0 + i) * ld + j;
            float f = 0.f;
            if (ok) {
              const float dv = v[hf * 8 + i] * (rj * ci.s);  // Delta V, scales undone exactly
              const float p = pb[i] + dv;                    // P = P_base + Delta V
              if (Pout) __stcs(Pout + o, p);
              if (prow) prow[cbase + c0 + i] = p;
              s_pv = fmaf(dv, dv, s_pv);
              float r;
              const float gap = gap2f(hj, lj, ci.hi, ci.lo);
              if (gap == 0.f && j != ic) flag_degenerate(a.st);
              map_entry<float>(z[i], p, ci.d, gap, j == ic, f, r);
              __stcs(Fout + o, f);
              if (oz) __stcs(oz + (int64_t)(cbase + c0 + i) * oz_ld + j, f);
              const float df = f - z[i];
              s_inc = fmaf(df, df, s_inc);
              s_z = fmaf(z[i], z[i], s_z);
              s_r = fmaf(r, r, s_r);
            }
            if (wn_h) {
              // V_next = F - Z_b(next) at the common scale, split (zero in padding);
              // this row's term of d_next = Delta_{cols[c], .} F_.c
              const float zb = zb_is_z ? z[i] : (zb_next ? zn[i] : (j == ic ? 1.f : 0.f));
              const float x = ok ? (f - zb) * sc_next : 0.f;
              uint16_t hh, ll;
              split16(x, a.fuse_bf16 != 0, hh, ll);
              __stcs(reinterpret_cast<unsigned short*>(wn_h) + o, (unsigned short)hh);
              if (wn_l) __stcs(reinterpret_cast<unsigned short*>(wn_l) + o, (unsigned short)ll);
              split_bad |= !(fabsf(x) <= split_max);
              dl[i] = ok ? dl[i] * f : 0.f;
            }
          }
          if (wn_h) {
            // column sums of the 8 terms over the warp's 32 rows (its row
            // group): lane L ends with column L / 4's sum (all four lanes of
            // each quad); every (column, group) partial is written once
            const float dsum = warp_colsum8(dl, lane);
            if ((lane & 3) == 0)
              a.dpart[(int64_t)(cbase + c0 + (lane >> 2)) * a.dgroups + grp] = (double)dsum;
          }
        }
      }
      tc_fence_before();
      if constexpr (PAIR) {
        // every lane's TMEM loads have completed; one release per warp to the first CTA
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(tempty_pair[acc]);
      } else {
        mbar_arrive(&ctl->tempty[acc]);
      }
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    if (split_bad) atomicOr(&a.st->split_bad, 1);
    // norm partials: warp sums, then one set of atomics per CTA (the slot of
    // this warp's column data is free once its last tile is done)
    const double b0 = warp_sum((double)s_inc), b1 = warp_sum((double)s_z),
                 b2 = warp_sum((double)s_r), b3 = warp_sum((double)s_pv);
    double* wsum = reinterpret_cast<double*>(ctl->wcol[e]);
    __syncwarp();
    if (lane == 0) {
      wsum[0] = b0;
      wsum[1] = b1;
      wsum[2] = b2;
      wsum[3] = b3;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");  // the epilogue warps only
    if (e == 0 && lane < 4) {
      double t = 0.0;
      for (int w = 0; w < EPI_WARPS; ++w) t += reinterpret_cast<double*>(ctl->wcol[w])[lane];
      double* dst = lane == 0 ? &a.st->acc_inc2
                              : lane == 1 ? &a.st->acc_z2 : lane == 2 ? &a.st->acc_r2
                                                                      : &a.st->acc_pv2;
      atomicAdd(dst, t);
    }
  }

  tc_fence_before();
  __syncthreads();
  // the peer may still load into / arrive on / multiply from this CTA until it is done
  if constexpr (CLUSTER) cluster_sync();
  tc_fence_after();
  if (warp == 1) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(TMEM_COLS)
                   : "memory");
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D 16-bit row-major [outer x inner] tensor, box [box_outer x 64], 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
              uint32_t box_outer, bool bf16) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
             const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

template <int MODE>
cudaError_t configure(int dev) {
  static int configured = -1;
  if (configured == dev) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes<MODE>());
  if (e == cudaSuccess) configured = dev;
  return e;
}

template <int MODE>
cudaError_t launch_cluster(const CUtensorMap& mDh, const CUtensorMap& mDl, const CUtensorMap& mWh,
                           const CUtensorMap& mWl, const CUtensorMap& mWh1,
                           const CUtensorMap& mWl1, const MapArgs<float>& a, int num_m, int num_n,
                           int num_kb, int passes, uint32_t idesc, int num_sms, cudaStream_t s) {
  static int max_clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // programmatic dependent launch: scheduled while the pre-pass finishes; the
  // kernel waits for it (griddep_wait) before it reads anything
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.blockDim = dim3(NUM_THREADS);
  cfg.dynamicSmemBytes = smem_bytes<MODE>();
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters <= 0) {
    // clusters that fit at once (one CTA per SM); pairs need two free SMs of a GPC
    cfg.gridDim = dim3(num_sms);
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, k_gemm_tc<MODE>, &cfg) != cudaSuccess || c <= 0)
      c = num_sms / 2;
    max_clusters = c;
  }
  const int pairs = (num_m / 2) * num_n;
  const int clusters = pairs < max_clusters ? pairs : max_clusters;
  cfg.gridDim = dim3(2 * clusters);
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_gemm_tc<MODE>, mDh, mDl, mWh, mWl, mWh1, mWl1, a, num_m,
                            num_n, num_kb,
                            passes, idesc);
}

cudaError_t launch_gemm_tc(const uint16_t* Dh, const uint16_t* Dl, const uint16_t* Wh,
                           const uint16_t* Wl, const MapArgs<float>& a, int npad, int kpad,
                           int passes, int bf16, int mode, cudaStream_t s) {
  if (npad % BM || kpad % BN || npad % BK || (passes != 1 && passes != 3))
    return cudaErrorInvalidValue;
  const bool bf = bf16 != 0;
  const int num_m = npad / BM, num_n = kpad / BN, num_kb = npad / BK;
  const bool pair = mode != IPT_PRODUCT_SINGLE && num_m % 2 == 0;
  CUtensorMap mDh, mDl, mWh, mWl, mWh1, mWl1;
  const uint32_t bbox = pair ? BN / 2 : BN;
  if (!make_map(&mDh, Dh, npad, npad, BM, bf) || !make_map(&mDl, Dl, npad, npad, BM, bf) ||
      !make_map(&mWh, Wh, npad, kpad, bbox, bf) || !make_map(&mWl, Wl, npad, kpad, bbox, bf))
    return cudaErrorInvalidValue;
  // the second W set (device-chosen operands with the next operand written by
  // the epilogue), else the first again
  const bool two = a.dyn && a.wnh[1] && a.wnl[1];
  if (!two) {
    mWh1 = mWh;
    mWl1 = mWl;
  } else if (!make_map(&mWh1, a.wnh[1], npad, kpad, bbox, bf) ||
             !make_map(&mWl1, a.wnl[1], npad, kpad, bbox, bf)) {
    return cudaErrorInvalidValue;
  }
  static int num_sms = 0, sms_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (sms_device != dev) {
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sms_device = dev;
  }
  if (pair) {
    if ((e = configure<MODE_PAIR>(dev)) != cudaSuccess) return e;
    return launch_cluster<MODE_PAIR>(mDh, mDl, mWh, mWl, mWh1, mWl1, a, num_m, num_n, num_kb,
                                     passes, idesc_for(bf, 2 * BM), num_sms, s);
  }
  if ((e = configure<MODE_SINGLE>(dev)) != cudaSuccess) return e;
  const int tiles = num_m * num_n;
  const int grid = tiles < num_sms ? tiles : num_sms;
  k_gemm_tc<MODE_SINGLE><<<grid, NUM_THREADS, smem_bytes<MODE_SINGLE>(), s>>>(
      mDh, mDl, mWh, mWl, mWh1, mWl1, a, num_m, num_n, num_kb, passes, idesc_for(bf, BM));
  return cudaGetLastError();
}

}  // namespace ipt
