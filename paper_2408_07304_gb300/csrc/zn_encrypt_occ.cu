// Hot path, register-capped launch shapes (kind 2): at most 128 registers per
// thread (512 threads' worth per SM) so that several blocks are resident on
// an SM and one block's memory and barrier phases overlap another's
// arithmetic; radix-16 passes.  2^10 <= N <= 2^13: one block per prime and
// ciphertext, 2^(LOGN-5) threads; N = 2^14: one block per output half of
// each limb (64 KiB of shared memory, 256 threads).
#include "zn_encrypt_kern.cuh"

namespace zn {

template <bool ZINC>
static cudaError_t enc_occ_dispatch(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  switch (P.log_n) {
    case 10: return enc_full<10, ZINC, 5, 16>(P, A, batch, st);
    case 11: return enc_full<11, ZINC, 5, 8>(P, A, batch, st);
    case 12: return enc_full<12, ZINC, 5, 4>(P, A, batch, st);
    case 13: return enc_full<13, ZINC, 5, 2>(P, A, batch, st);
    case 14: return enc_half<13, ZINC, 5, 2>(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_encrypt_occ(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return zinc ? enc_occ_dispatch<true>(P, A, batch, st) : enc_occ_dispatch<false>(P, A, batch, st);
}

}  // namespace zn
