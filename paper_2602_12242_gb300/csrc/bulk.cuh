// Bulk (non-tensor) asynchronous copies between global and shared memory
// (cp.async.bulk): loads complete on an mbarrier through its transaction
// count, stores form bulk groups of the issuing thread.  Every wait is
// bounded; a wait that runs out returns false and the caller records the
// failure instead of spinning on.
//
// Rules the callers keep: addresses and sizes are multiples of 16 bytes; a
// phase's transaction count stays below 2^20 bytes; shared memory written by
// ordinary stores is fenced (fence_proxy_async_smem) by the writing threads
// before a barrier and the bulk store that reads it.
#pragma once

#include <stdint.h>

namespace mx {

constexpr unsigned long long kBulkWaitNs = 1000000000ull;  // a wait gives up after about one second
constexpr int kBulkWaitPolls = 1 << 26;                        // and after this many polls in any case

__device__ __forceinline__ uint32_t smem_u32addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier ordinary shared-memory accesses before later
// bulk-copy (async proxy) accesses of the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32addr(bar)), "r"(bytes)
               : "memory");
}

// global -> shared, completes `bytes` transactions on `bar`
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32addr(dst_smem)),
               "l"(src), "r"(bytes), "r"(smem_u32addr(bar))
               : "memory");
}

// shared -> global, in the issuing thread's current bulk group
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32addr(src_smem)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// this thread's bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// this thread's bulk stores are complete; their global writes are ordered
// before this thread's later ordinary accesses
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the completion of phase `parity` of `bar`: false after
// about kBulkWaitNs of global time (checked every 256 polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32addr(bar);
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < kBulkWaitPolls; ++i) {
    if ((i & 255) == 255 && global_ns() - t0 > kBulkWaitNs) return false;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

}  // namespace mx
