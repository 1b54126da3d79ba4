// Tensor memory (TMEM) as per-thread parking space for the encryption
// epilogues: the vanilla shape (Eq. 8) needs u-hat = NTT(u) again in the
// epilogues of the two later transforms, and a 256-thread CTA that owns
// 2^13 outputs has no shared memory left beside its transform buffer.
//
// Layout: a CTA allocates 128 columns (128 lanes x 128 x 32-bit words =
// 64 KiB).  Warp w accesses the lane quarter 32 (w mod 4) (the tcgen05.ld /
// tcgen05.st lane rule); warps w and w + 4 take columns [0, 64) and
// [64, 128).  Thread t keeps its i-th epilogue output (index t + 256 i of the
// staged epilogue, i < 32) in columns 2i, 2i + 1 of its lane: 32 words of 64
// bits, exactly one 2^13-residue quarter per CTA.
//
// Allocation never waits: every kernel that allocates here requests 128
// columns and holds at least 64 KiB of dynamic shared memory, so at most
// three such CTAs share an SM (228 KiB), i.e. 384 of the 512 columns.
#pragma once
#include "zn_kernels.h"

namespace zn {
namespace tmem {

constexpr unsigned kCols = 128;
constexpr size_t kMinSmemPerCta = 64 * 1024;
static_assert(4 * kMinSmemPerCta > 228 * 1024, "at most three TMEM-holding CTAs per SM");
static_assert(3 * kCols <= 512, "three CTAs' columns fit in one SM's tensor memory");

// One full warp (convergent); writes the base address into *slot and gives
// up the CTA's right to allocate again.
__device__ __forceinline__ void alloc(unsigned* slot) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(slot);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(kCols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// One full warp, after every thread's last access (fence + barrier first).
__device__ __forceinline__ void dealloc(unsigned base) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(kCols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// This thread's lane and column base (warp-uniform apart from the lane the
// hardware adds per thread).
__device__ __forceinline__ unsigned thread_base(unsigned base) {
  const unsigned w = threadIdx.x >> 5;
  return base + (((w & 3u) * 32u) << 16) + (w >> 2) * 64u;
}

// 64-bit word into two columns of this thread's lane (whole warp, the same
// column for every lane).
__device__ __forceinline__ void st_u64(unsigned addr, u64 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(addr), "r"((unsigned)v),
               "r"((unsigned)(v >> 32)));
}

// The word back (waits for the load).
__device__ __forceinline__ u64 ld_u64(unsigned addr) {
  unsigned lo, hi;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(lo), "=r"(hi)
      : "r"(addr));
  return ((u64)hi << 32) | lo;
}

// This thread's stores have completed (before its later loads of them).
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Parking for a 256-thread staged epilogue over 2^13 outputs: thread t is
// handed the indices t + 256 i (i < 32), and i picks the columns.
struct Park {
  unsigned a;     // thread_base of the CTA's allocation
  __device__ __forceinline__ void put(int idx, u64 v) const { st_u64(a + 2u * (unsigned)(idx >> 8), v); }
  __device__ __forceinline__ u64 get(int idx) const { return ld_u64(a + 2u * (unsigned)(idx >> 8)); }
  __device__ __forceinline__ void done() const { wait_st(); }
};

// The allocation around a kernel body: warp 0 allocates, every thread sees
// the address; at the end warp 0 frees it after every thread is done.  The
// warp test goes through a shuffle so that the compiler sees it as uniform
// per warp (with threadIdx.x < 32 the N = 2^15 vanilla kernel spilled 44
// bytes at 80 registers; with this test it spills none).
struct Scope {
  unsigned base;
  __device__ __forceinline__ explicit Scope(unsigned* slot) {
    if (__shfl_sync(0xffffffffu, threadIdx.x >> 5, 0) == 0) alloc(slot);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    base = *slot;
  }
  // every thread's loads have completed (ld_u64 waits); the fence pair
  // around the barrier orders them before the free
  __device__ __forceinline__ void release() const {
    fence_before_sync();
    __syncthreads();
    if (__shfl_sync(0xffffffffu, threadIdx.x >> 5, 0) == 0) {
      fence_after_sync();
      dealloc(base);
    }
  }
};

}  // namespace tmem
}  // namespace zn
