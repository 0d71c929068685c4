// ipt_residual_dense_noalloc: the FP64 residual ||M Z - Z Lambda||_F computed
// without any device allocation.
//
// Who needs this: code that must not call cudaMalloc -- processes whose
// device memory is owned by another allocator (a framework's caching pool, a
// fixed memory budget) that forbids side allocations, and latency-critical
// loops where cudaMalloc / cudaFree would synchronise the device.  The
// solver's own verification path converts M and Z into handle-allocated FP64
// copies and accumulates into an allocated scalar; this variant reads the
// caller's M and Z in place (FP64 or FP32) and keeps its only scratch -- one
// FP64 partial sum per thread block -- in a fixed-size file-scope device array
// that lives as long as the library is loaded.
#include <math.h>
#include <mutex>

#include "ipt_internal.cuh"

namespace {

constexpr int TILE = 64;                   // outputs per block: TILE x TILE
constexpr int NOALLOC_MAX_BLOCKS = 16384;  // scratch capacity: partial sums

// The scratch: one partial sum of squared residual entries per block.
// Every call overwrites the slots of the blocks it launches before the final
// sum reads them, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS];

__device__ __forceinline__ double load_elem(const void* p, int64_t idx, int dtype) {
  return dtype == IPT_DTYPE_F64 ? static_cast<const double*>(p)[idx]
                                : static_cast<double>(static_cast<const float*>(p)[idx]);
}

// Block (bx, by) computes R = M Z - Z Lambda on rows [64 by, +64) and columns
// [64 bx, +64) with a 16x16 thread grid (4x4 outputs each, FP64 FMA), and
// stores the sum of R^2 over its tile into partials[by * gridDim.x + bx].
__global__ void __launch_bounds__(256)
    k_residual_noalloc(int n, int k, const void* __restrict__ M, int64_t ldm, int m_dtype,
                       const void* __restrict__ Z, int64_t ldz, int z_dtype,
                       const double* __restrict__ lambda, double* __restrict__ partials) {
  __shared__ double As[8][TILE + 1];
  __shared__ double Bs[8][TILE + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * TILE;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 8) {
    // 64x8 tiles of M (rows r0.., cols k0..) and of Z^T (cols c0.., rows k0..)
    for (int e = tid; e < TILE * 8; e += 256) {
      const int rr = e >> 3, kk = e & 7;
      const int gr = r0 + rr, gk = k0 + kk, gc = c0 + rr;
      As[kk][rr] = (gr < n && gk < n) ? load_elem(M, (int64_t)gr * ldm + gk, m_dtype) : 0.0;
      Bs[kk][rr] = (gc < k && gk < n) ? load_elem(Z, (int64_t)gc * ldz + gk, z_dtype) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (r < n && c < k) {
        const double res = acc[i][j] - load_elem(Z, (int64_t)c * ldz + r, z_dtype) * lambda[c];
        s += res * res;
      }
    }
  }
  s = ipt::warp_sum(s);
  __shared__ double red[8];
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partials[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// One block: sum the partials in a fixed order and write the norm.
__global__ void k_residual_noalloc_final(const double* __restrict__ partials, int count,
                                         double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

// Device address of the scratch array, looked up once per device and CUDA
// context (a cudaDeviceReset ends the context the cached address belongs to;
// the next call sees a new context id and looks the address up again).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

std::mutex g_mu;
double* g_ptr[64] = {};
unsigned long long g_ctx[64] = {};

// Id of the current context (0 if the driver cannot tell).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<CtxGetCurrentFn>(a);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(b);
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
  return 0;
}

ipt_status scratch_for_current_device(double** ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return IPT_CUDA_ERROR;
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_ptr[dev] || g_ctx[dev] != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p)
      return IPT_CUDA_ERROR;
    g_ptr[dev] = static_cast<double*>(p);
    g_ctx[dev] = ctx;
  }
  *ptr = g_ptr[dev];
  return IPT_OK;
}

}  // namespace

extern "C" ipt_status ipt_residual_dense_noalloc(int64_t n, const void* M, int64_t ldm,
                                                 int m_dtype, int64_t k, const void* Z,
                                                 int64_t ldz, int z_dtype, const double* lambda,
                                                 double* out, void* stream) {
  if (!M || !Z || !lambda || !out || n < 1 || k < 1 || k > n || ldm < n || ldz < n)
    return IPT_INVALID_ARG;
  if ((m_dtype != IPT_DTYPE_F64 && m_dtype != IPT_DTYPE_F32) ||
      (z_dtype != IPT_DTYPE_F64 && z_dtype != IPT_DTYPE_F32))
    return IPT_INVALID_ARG;
  const int64_t bx = (k + TILE - 1) / TILE, by = (n + TILE - 1) / TILE;
  if (bx * by > NOALLOC_MAX_BLOCKS) return IPT_UNSUPPORTED;  // beyond the fixed scratch
  // an error left by earlier work stays the caller's to read: report it without
  // launching and without clearing it
  if (cudaPeekAtLastError() != cudaSuccess) return IPT_CUDA_ERROR;
  double* partials = nullptr;
  ipt_status st = scratch_for_current_device(&partials);
  if (st != IPT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid((unsigned)bx, (unsigned)by);
  k_residual_noalloc<<<grid, 256, 0, s>>>((int)n, (int)k, M, ldm, m_dtype, Z, ldz, z_dtype,
                                          lambda, partials);
  k_residual_noalloc_final<<<1, 256, 0, s>>>(partials, (int)(bx * by), out);
  return cudaGetLastError() == cudaSuccess ? IPT_OK : IPT_CUDA_ERROR;
}
