// Bulk asynchronous copies (global -> shared, the TMA engine's linear mode)
// completed on shared-memory mbarriers, in inline PTX for sm_100-family GPUs.
//
// A copy is issued by one thread: mbarrier.arrive.expect_tx announces the
// bytes, cp.async.bulk moves them and signals the barrier's transaction
// count; the barrier's phase completes when all bytes have landed.  Every
// wait is bounded: a caller that sees `false` treats the copy as lost.
#pragma once

#include <cstdint>

namespace mdhp {

// try_wait polls (each poll may suspend the thread for a short, hardware-chosen
// time); 1 << 22 polls is far beyond any copy's latency.
constexpr uint32_t kWaitPolls = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// makes initialised barriers visible to the async proxy (the copy engine)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// bytes and both addresses multiples of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false after kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// A consumer's wait with a caller-chosen bound: polls = 0 is mbar_wait;
// otherwise at most `polls` non-blocking tests (a plan can shorten the
// consumers' waits to exercise the timeout path; the drains that make a
// CTA's shared memory safe to reuse always take the full bound).
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, uint32_t polls) {
  if (polls == 0) return mbar_wait(bar, parity);
  for (uint32_t i = 0; i < polls; ++i)
    if (mbar_test_wait(bar, parity)) return true;
  return false;
}

// generic-proxy stores to global memory -> visible to later bulk copies
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// generic-proxy accesses of shared memory ordered before later bulk copies
// into it (a ring slot read by threads, then refilled by the copy engine)
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace mdhp
