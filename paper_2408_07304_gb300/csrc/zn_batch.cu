// Mixed rings in one persistent launch: k_batch_encrypt walks a work list of
// packets (same-ring units filling a 512-thread block) across rings of
// different degree, chain and mode.  The unit code lives in
// zn_encrypt_unit.cuh.
#include "zn_encrypt_unit.cuh"

namespace zn {

// -------------------------------------------------- mixed rings, persistent

// Packet: `count` units of one job -- ciphertexts b0 .. b0+count-1 at prime
// `prime` (half `half` for N = 2^15) -- processed together by one 512-thread
// block, 2^(LOGN-5) threads and 2^LOGN shared words per unit.
// __noinline__: each ring size is register-allocated on its own instead of
// the kernel carrying the union of every path's registers.
template <int LOGN, bool ZINC>
__device__ __noinline__ void batch_full(const JobDesc& J, const EncPacket& pk, u64* sm) {
  using S = NttShape<LOGN, 5>;
  const int g = threadIdx.x / S::T, t = threadIdx.x % S::T;
  encrypt_unit<LOGN, ZINC, 5>(J.P, J.E, pk.prime, (size_t)pk.b0 + g, sm + (size_t)g * S::N, t, g < (int)pk.count);
}

template <bool ZINC>
__device__ __noinline__ void batch_half(const JobDesc& J, const EncPacket& pk, u64* sm) {
  encrypt_half_unit<14, ZINC, 5>(J.P, J.E, pk.prime, pk.half, pk.b0, sm, threadIdx.x);
}

template <bool ZINC>
__device__ __forceinline__ void batch_packet(const JobDesc& J, const EncPacket& pk, u64* sm) {
  switch (J.P.log_n) {
    case 10: batch_full<10, ZINC>(J, pk, sm); break;
    case 11: batch_full<11, ZINC>(J, pk, sm); break;
    case 12: batch_full<12, ZINC>(J, pk, sm); break;
    case 13: batch_full<13, ZINC>(J, pk, sm); break;
    case 14: batch_full<14, ZINC>(J, pk, sm); break;
    case 15: batch_half<ZINC>(J, pk, sm); break;
    default: break;
  }
}

// Persistent: one 512-thread block per SM; each block takes the next packet
// from a global counter until the list is exhausted (no block waits for any
// other).  The counter must be zero at launch.
__global__ void __launch_bounds__(512, 1) k_batch_encrypt(const JobDesc* __restrict__ jobs,
                                                          const EncPacket* __restrict__ packets, int n_packets,
                                                          int* counter) {
  extern __shared__ u64 sm[];
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int p = s_next;
    __syncthreads();
    if (p >= n_packets) break;
    const EncPacket pk = packets[p];
    const JobDesc& J = jobs[pk.job];
    if (J.zinc) batch_packet<true>(J, pk, sm);
    else batch_packet<false>(J, pk, sm);
    __syncthreads();
  }
}

cudaError_t batch_encrypt_attributes() {
  return cudaFuncSetAttribute(k_batch_encrypt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(u64) << 14));
}

// Capturable: the attribute is set beforehand by batch_set_attributes().
cudaError_t launch_batch_encrypt(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter, int grid,
                                 cudaStream_t st) {
  k_batch_encrypt<<<grid, 512, sizeof(u64) << 14, st>>>(jobs, packets, n_packets, counter);
  return cudaGetLastError();
}

}  // namespace zn
