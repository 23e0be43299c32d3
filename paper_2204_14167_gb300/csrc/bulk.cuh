// Bulk asynchronous copies (the TMA engine's untiled form) from global into
// shared memory, completing on an mbarrier, and the bounded waits on them.
//
// A copy is issued by one thread: mbarrier.arrive.expect_tx announces the
// byte count, cp.async.bulk moves the bytes and signals completion on the
// same barrier.  Both addresses must be 16-byte aligned and the size a
// multiple of 16.  Every wait polls at most BULK_WAIT_POLLS times, so that a
// copy that never lands ends the kernel with an error flag instead of a hang.
#pragma once
#include <cstdint>

namespace discos {

constexpr int BULK_WAIT_POLLS = 1 << 20;
// Fault-word bit set by a kernel whose bounded wait on an asynchronous copy
// ran out.
constexpr unsigned FAULT_ASYNC_WAIT = 8u;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (and those made
// visible to it by a CTA barrier) before later asynchronous-proxy writes.
__device__ __forceinline__ void async_proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copies `bytes` from global src to shared dst; completion arrives on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Waits for the completion of phase `parity` of bar; false if it did not
// complete within BULK_WAIT_POLLS polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < BULK_WAIT_POLLS; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace discos
