// Thread-block cluster helpers shared by the cluster encryption kernels (the
// N = 2^15 four-CTA quarters, zn_quarter.cuh, and the N = 2^14 two-CTA
// halves, zn_pair.cuh): the CTA's rank, a cluster-wide barrier, stores into
// another CTA's shared memory (distributed shared memory, this GPU only; no
// multicast), and the launch with a cluster dimension.
#pragma once
#include "zn_kernels.h"

namespace zn {
namespace cluster {

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster; release / acquire order the
// shared-memory accesses before the barrier against those after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory address of `p` in the CTA of cluster rank `rank`.
__device__ __forceinline__ unsigned map_rank(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster(unsigned addr, u64 v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// Harvey keeps [0, 4q); a relaxed stage adds 2q: the generators bring their
// outputs back below 4q so that the 12 local stages end below 28q.
template <bool RELAX>
__device__ __forceinline__ u64 below4q(u64 x, u64 q) {
  if constexpr (RELAX) return x >= 4 * q ? x - 4 * q : x;
  return x;
}

// Launch `kern` with clusters of `size` consecutive CTAs along x, `threads`
// per CTA and `smem` bytes of dynamic shared memory.
template <class... Args>
cudaError_t launch(unsigned size, size_t smem, void (*kern)(Args...), dim3 grid, unsigned threads, cudaStream_t st,
                   Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace cluster
}  // namespace zn
