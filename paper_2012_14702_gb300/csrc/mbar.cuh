// Shared-memory barrier primitives and the bounded wait used by the
// tensor-core product kernel (k_tc_gemm.cu) and by the bounded-wait check
// (k_diag.cu).  Every wait gives up after a time limit read from
// %globaltimer, so a barrier that is never completed ends in an error status
// instead of a hung GPU.
#pragma once

#include <cstdint>

namespace ipt {
namespace mbar {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: far above any legitimate wait

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same test with cluster-scope acquire: for barriers that threads of the
// peer CTA arrive on.
__device__ __forceinline__ bool mbar_try_cluster(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase `parity` of barrier b.  False on timeout or when another
// role has aborted (then the caller stops issuing and falls through to drain).
template <bool CLUSTER = false>
__device__ __noinline__ bool wait_bounded(uint64_t* b, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = kWaitLimitNs) {
  auto test = [&]() { return CLUSTER ? mbar_try_cluster(b, parity) : mbar_try(b, parity); };
  if (test()) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (test()) return true;
    if (*abort) return false;
    if (gtimer() - t0 > limit_ns) return false;
  }
}
}  // namespace mbar
}  // namespace ipt
