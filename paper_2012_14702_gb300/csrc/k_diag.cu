// Checks of device-side building blocks, without any fault or hang.
//
// Bounded-wait check: exercises the give-up path of the shared-memory barrier
// wait that every waiting role of the tensor-core product kernel uses, without
// any fault or hang.  One CTA; thread 0 initialises a barrier for one arrival
// and waits on its first phase with a caller-given limit.  With `arrive` a
// thread of the second warp arrives and the wait must succeed; without it
// nothing ever arrives and the wait must give up once the limit has passed.
#include "ipt_internal.cuh"
#include "mbar.cuh"

namespace ipt {

namespace {

__global__ void k_wait_check(int arrive, uint64_t limit_ns, long long* out) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar::mbar_init(&bar, 1);
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 32 && arrive) mbar::mbar_arrive(&bar);
  if (threadIdx.x == 0) {
    const uint64_t t0 = mbar::gtimer();
    const bool ok = mbar::wait_bounded(&bar, 0u, &abort_flag, limit_ns);
    out[0] = ok ? 1 : 0;
    out[1] = (long long)(mbar::gtimer() - t0);
  }
}

// The FP32 map's division u / gap as the epilogues compute it (u times the
// refined reciprocal), one entry per thread.
__global__ void k_recip_check(int64_t count, const float* __restrict__ gap,
                              const float* __restrict__ u, float* __restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) q[i] = u[i] * recip_nr(gap[i]);
}

// The integer-ALU conversions of the sparse setup pass, one entry per thread.
__global__ void k_conv_check(int64_t count, const double* __restrict__ x, float* __restrict__ hi,
                             float* __restrict__ lo, float* __restrict__ f,
                             double* __restrict__ back, int32_t* __restrict__ ok) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  bool a, b, c;
  float h, l;
  split_f64_bits(x[i], h, l, a);
  const float r = f64_to_f32_rn_bits(x[i], b);
  const double d = f32_to_f64_bits(r, c);
  hi[i] = h;
  lo[i] = l;
  f[i] = r;
  back[i] = d;
  ok[i] = (a ? 1 : 0) | (b ? 2 : 0) | (c ? 4 : 0);
}

}  // namespace

cudaError_t launch_conv_check(int64_t count, const double* x, float* hi, float* lo, float* f,
                              double* back, int32_t* ok, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_conv_check<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, x, hi, lo, f, back, ok);
  return cudaGetLastError();
}

cudaError_t launch_recip_check(int64_t count, const float* gap, const float* u, float* q,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_recip_check<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, gap, u, q);
  return cudaGetLastError();
}

cudaError_t launch_wait_check(int arrive, uint64_t limit_ns, long long* out, cudaStream_t s) {
  k_wait_check<<<1, 64, 0, s>>>(arrive, limit_ns, out);
  return cudaGetLastError();
}

}  // namespace ipt
