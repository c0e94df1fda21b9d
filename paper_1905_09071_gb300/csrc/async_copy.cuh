// Bulk asynchronous global->shared copies (the TMA engine's non-tensor form)
// completed through a shared-memory mbarrier, with bounded waits.
//
// cp.async.bulk moves `bytes` (a multiple of 16, 16-byte aligned on both
// sides) and signals the transaction count on the mbarrier; a waiter spins on
// the mbarrier's phase parity. Every wait here gives up after `limit` clock
// cycles and reports that instead of hanging.
#pragma once

#include <cstdint>

namespace sag {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals)
               : "memory");
}

// Makes the initialised barriers visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Drops the 128-byte L2 line at p (128-byte aligned) without writing it
// back: for workspace data that no kernel reads again.
__device__ __forceinline__ void discard_l2(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Clock cycles a block that gave up waiting still waits for its own copies in
// flight before it exits (about 2 s at the maximum SM clock).
constexpr long long kDrainLimit = 4000000000LL;

// Waits for phase `parity` of the barrier; false if `limit` cycles pass first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// A block whose wait gave up: latch the timeout status, then let the copies
// it has in flight on `bar` (phase `parity`) land before it exits. If that
// second wait also runs out, the block exits with copies still in flight into
// shared memory a later block may reuse, so `undrained_bit` is latched as
// well and the host reports the context as suspect. Called by one thread; out
// of line, as it runs at most once.
static __device__ __noinline__ void timeout_drain(unsigned* status, unsigned bit, unsigned undrained_bit,
                                                  uint64_t* bar, uint32_t parity) {
  atomicOr(status, bit);
  if (!mbar_wait_bounded(bar, parity, kDrainLimit)) atomicOr(status, undrained_bit);
}

}  // namespace sag
