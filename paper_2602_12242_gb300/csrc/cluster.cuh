// Thread-block cluster helpers (inline PTX): the CTA's rank in its cluster,
// a cluster-wide barrier, and the address of the same shared-memory location
// in another CTA of the cluster (distributed shared memory).
#pragma once

#include <stdint.h>

namespace mx {

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster arrives (release) and waits
// (acquire): shared-memory writes before it are visible to the other CTAs
// after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Split form: arrive (no memory ordering) now, wait later.  A CTA that has
// passed cluster_wait() knows every CTA of the cluster has started, so their
// shared memory may be written through cluster_map() addresses.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

// Split form with memory ordering: this thread's earlier memory accesses
// (shared memory of any CTA of the cluster included) are performed before the
// arrive, and accesses after the wait see what the other threads released.
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// generic address of the same shared-memory location in CTA `rank` of the cluster
template <typename T> __device__ __forceinline__ const T* cluster_map(const T* p, unsigned rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
  return reinterpret_cast<const T*>(out);
}

}  // namespace mx
