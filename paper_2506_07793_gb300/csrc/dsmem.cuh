// dsmem.cuh -- thread-block-cluster primitives in inline PTX (sm_90 and up):
// this CTA's rank in its cluster, the cluster barrier, and a load from the
// same shared-memory offset in another CTA of the cluster (distributed shared
// memory).  No header of the toolkit, so that the plan-time compiler
// (jit.cu) builds the kernels that use it.
#pragma once

namespace cwtk {

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster arrives; shared-memory writes before
// the barrier (release) are visible to the cluster's reads after it (acquire).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Load a float2 from the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ float2 ld_cluster(const float2 *local, unsigned rank) {
    const unsigned laddr = (unsigned)__cvta_generic_to_shared(local);
    unsigned raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(raddr) : "memory");
    return v;
}

}  // namespace cwtk
