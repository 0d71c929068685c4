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
// The tensor-core variant (BF16 products) is k_batched_tc.cu.
#include "ipt_internal.cuh"

namespace ipt {

namespace {

constexpr int TB = 64;   // largest output tile (rows and columns)
constexpr int TK = 32;   // product depth per shared-memory stage
constexpr int NT = 256;  // threads per CTA (16 x 16, 4 x 4 outputs each)
constexpr int kU = 8;    // loads in flight per thread in the per-problem passes

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

__global__ void __launch_bounds__(NT, 3) k_batched(BatchArgs a) {
  __shared__ Shared sh;
  const int tid = threadIdx.x;
  float* z0 = a.scratch + (int64_t)blockIdx.x * 2 * a.max_n2;
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
    double r0 = 0.0;
    int status = IPT_MAXITER, it = 0;
    // ---------------------------------------------------------- evaluations
    for (it = 0; it < a.max_iter; ++it) {
      // FP32 per-thread sums, CTA sums as FP32 pairs and the test in FP64 on
      // one thread (the FP64 pipe runs at a small fraction of the FP32 rate
      // here, so no per-entry or per-thread FP64 work)
      float s_inc = 0.f, s_z = 0.f, s_r = 0.f;
      if (it == 0) {
        // Z = E: product-free.  Entries in the iterate's storage order, kU
        // loads in flight per thread before their use.
        const int n2 = n * n;
        for (int base = tid; base < n2; base += kU * NT) {
          float dl[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int e = base + u * NT, j = e / n, c = e % n;
            dl[u] = e < n2 ? M[(int64_t)j * n + c] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int e = base + u * NT, j = e / n, c = e % n;
            if (e >= n2) continue;
            const float djc = dl[u];
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
            zn[e] = f;
          }
        }
        s_z = tid == 0 ? (float)n : 0.f;
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
    const int n2 = n * n;  // over Zout's column-major order, kU loads in flight
    for (int base = tid; base < n2; base += kU * NT) {
      float v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = base + u * NT;
        v[u] = (e < n2 && !is_e) ? zc[(int64_t)(e % n) * n + e / n] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = base + u * NT;
        if (e < n2) Zout[e] = is_e ? ((e / n == e % n) ? 1.f : 0.f) : v[u];
      }
    }
    for (int c = tid; c < n; c += NT) {
      const double t = a.theta ? a.theta[vo + c] : (double)M[(int64_t)c * n + c];
      a.lambda[vo + c] = t + (double)sh.d[c];
    }
    if (tid == 0) {
      a.status[p] = status;
      a.iters[p] = evals;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_batched(const float* M, const double* theta, const int64_t* m_off,
                           const int64_t* v_off, const int* nsz, const int* order, int count,
                           int64_t max_n2, double tol, int max_iter, int stop,
                           double diverge_bound, double* lambda, float* Z, int* status,
                           int* iters, float* scratch, int* queue, const int* tiles, int ctas,
                           cudaStream_t s) {
  BatchArgs a;
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
  k_batched<<<ctas, NT, 0, s>>>(a);
  return cudaGetLastError();
}

int batched_ctas_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched, NT, 0) != cudaSuccess ||
      nb < 1)
    nb = 1;
  return nb;
}

}  // namespace ipt
