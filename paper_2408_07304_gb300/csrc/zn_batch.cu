// Mixed rings in persistent launches: k_batch_encrypt3 walks the work list of
// rings up to 2^13 (three 256-thread blocks per SM), across rings of
// different degree, chain and mode; the lists of 2^14 and 2^15 rings run on
// persistent two- and four-CTA clusters (zn_encrypt_pair.cu,
// zn_encrypt_quarter.cu).  The unit code lives in zn_encrypt_unit.cuh.
#include "zn_encrypt_unit.cuh"

namespace zn {

// --------------------------------- rings up to 2^14, three blocks per SM
// 256-thread blocks with 80 registers and 64 KiB of shared memory, so that
// three share an SM (the radix-8 units of the single-ring kind 3): 2^13 one
// limb per block, smaller rings 2^(13 - LOGN) limbs per block.

template <int LOGN, bool ZINC>
__device__ __noinline__ void batch3_full(const JobDesc& J, const EncPacket& pk, u64* sm) {
  using S = NttShape<LOGN, 5>;
  const int g = threadIdx.x / S::T, t = threadIdx.x % S::T;
  encrypt_unit<LOGN, ZINC, 5, 3>(J.P, J.E, pk.prime, (size_t)pk.b0 + g, sm + (size_t)g * S::N, t, g < (int)pk.count);
}

template <bool ZINC>
__device__ __forceinline__ void batch3_packet(const JobDesc& J, const EncPacket& pk, u64* sm) {
  switch (J.P.log_n) {
    case 10: batch3_full<10, ZINC>(J, pk, sm); break;
    case 11: batch3_full<11, ZINC>(J, pk, sm); break;
    case 12: batch3_full<12, ZINC>(J, pk, sm); break;
    case 13: batch3_full<13, ZINC>(J, pk, sm); break;
    default: break;
  }
}

__global__ void __launch_bounds__(256, 3) k_batch_encrypt3(const JobDesc* __restrict__ jobs,
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
    if (J.zinc) batch3_packet<true>(J, pk, sm);
    else batch3_packet<false>(J, pk, sm);
    __syncthreads();
  }
}

cudaError_t batch_encrypt_attributes() {
  cudaError_t e = batch_quarter_attributes();
  if (e != cudaSuccess) return e;
  if ((e = batch_pair_attributes()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_batch_encrypt3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(u64) << 13));
}

// Capturable: the attributes are set beforehand by batch_set_attributes().
// The list of rings up to 2^13 on three 256-thread blocks per SM.
cudaError_t launch_batch_encrypt(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter, int sms,
                                 cudaStream_t st) {
  k_batch_encrypt3<<<3 * sms, 256, sizeof(u64) << 13, st>>>(jobs, packets, n_packets, counter);
  return cudaGetLastError();
}

}  // namespace zn
