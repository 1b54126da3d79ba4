// Register-capped launch shapes (kind 3): at most 80 registers per thread
// (768 threads' worth per SM, three blocks of 256 threads) with radix-8
// passes, which need fewer live registers than radix-16 ones.  2^10 <= N <=
// 2^13: one block per prime and ciphertext, 2^(LOGN-5) threads.  (Kind 3 at
// N = 2^14 and 2^15 runs the cluster kernels, zn_encrypt_pair.cu and
// zn_encrypt_quarter.cu.)
#include "zn_encrypt_kern.cuh"

namespace zn {

template <bool ZINC>
static cudaError_t enc_occ3_dispatch(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  switch (P.log_n) {
    case 10: return enc_full<10, ZINC, 5, 24, 3>(P, A, batch, st);
    case 11: return enc_full<11, ZINC, 5, 12, 3>(P, A, batch, st);
    case 12: return enc_full<12, ZINC, 5, 6, 3>(P, A, batch, st);
    case 13: return enc_full<13, ZINC, 5, 3, 3>(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_encrypt_occ3(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return zinc ? enc_occ3_dispatch<true>(P, A, batch, st) : enc_occ3_dispatch<false>(P, A, batch, st);
}

}  // namespace zn
