// Bulk asynchronous copies (the TMA engine's untiled form) from global to shared memory,
// completed on shared-memory mbarriers, and a bounded wait on them.
//
// Rules the callers keep:
//   * source and destination addresses are 16-byte aligned and the size is a multiple of
//     16 bytes (cp.async.bulk);
//   * one thread arms a barrier (arrive + expected transaction bytes) and issues the copy
//     that completes it; every consumer waits on the barrier's phase parity;
//   * a slot is refilled only after every consumer has read it: each consumer fences the
//     async proxy after its reads, the warp synchronises, then one thread issues the refill;
//   * no wait is unbounded: mbar_wait_bounded gives up after kBulkWaitNs of global time, and
//     the caller then records a timeout in the device status word, drains its own copies in
//     flight with the same bound, and returns.
#pragma once
#include <cstdint>

namespace numa_dev {

// A wait gives up after this much global time (a legitimate wait lasts microseconds).
constexpr unsigned long long kBulkWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses (barrier initialisation,
// reads of a slot about to be refilled, writes a bulk store will read) before later
// async-proxy (bulk copy) accesses.  Every thread that touched the memory fences, then the
// threads synchronise, then one thread issues the copy.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive once on the barrier and add `bytes` to the transaction count it waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Copy `bytes` from global memory to this CTA's shared memory; completion is signalled as
// transaction bytes on the barrier.
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
      : "memory");
}

// Copy `bytes` from this CTA's shared memory to global memory (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* dst, unsigned src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                   (unsigned long long)__cvta_generic_to_global(dst)),
               "r"(src), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every committed bulk store of this thread has finished reading shared memory
// (a hardware wait on the thread's own copies; it needs no bound).
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false after kBulkWaitNs (or 2^24
// polls, whichever comes first).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < (1u << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kBulkWaitNs) return false;
  }
  return false;
}

}  // namespace numa_dev
