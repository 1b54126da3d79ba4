// Hot path, one ring per launch, and the launch-shape dispatch.  Kind 0 (this
// file): k_encrypt (N <= 2^14, one block per prime and ciphertext) and
// k_encrypt_half (N = 2^15, two blocks per prime and ciphertext).  Kind 1:
// the multi-polynomial kernel (zn_encrypt_mp.cu).  Kinds 2 and 3:
// register-capped shapes with two or three resident blocks per SM
// (zn_encrypt_occ.cu, zn_encrypt_occ3.cu).
#include "zn_encrypt_kern.cuh"

namespace zn {

// ------------------------------------------------------- one ring per launch

// variant = 2 * kind + order; order 0 prime-major, 1 ciphertext-major.  Kind
// 1 applies for 2^10 <= N <= 2^14 with 16-byte aligned key, companion and
// output pointers, kind 2 for 2^10 <= N <= 2^14, kind 3 for 2^10 <= N <= 2^15
// (at 2^14 the two-CTA cluster kernel, zn_encrypt_pair.cu, at 2^15 the
// four-CTA one, zn_encrypt_quarter.cu); otherwise kind 0 runs.
template <bool ZINC>
static cudaError_t enc_dispatch(const DevParams& P, const EncArgs& A_in, uint32_t batch, int variant,
                                cudaStream_t st) {
  EncArgs A = A_in;
  A.swap = variant & 1;
  const int kind = variant >> 1;
  if (kind == 1 && P.log_n >= 10 && P.log_n <= 14 && aligned16(A.key) && aligned16(A.out) &&
      (ZINC || aligned16(A.keys)))
    return launch_encrypt_mp(P, A, ZINC, batch, st);
  if (kind == 2 && P.log_n >= 10 && P.log_n <= 14) return launch_encrypt_occ(P, A, ZINC, batch, st);
  if (kind == 3 && P.log_n == 14) return launch_encrypt_pair(P, A, ZINC, batch, st);
  if (kind == 3 && P.log_n >= 10 && P.log_n <= 13) return launch_encrypt_occ3(P, A, ZINC, batch, st);
  if (kind == 3 && P.log_n == 15) return launch_encrypt_quarter(P, A, ZINC, batch, st);
  switch (P.log_n) {
    case 4: return enc_full<4, ZINC, 5>(P, A, batch, st);
    case 5: return enc_full<5, ZINC, 5>(P, A, batch, st);
    case 6: return enc_full<6, ZINC, 5>(P, A, batch, st);
    case 7: return enc_full<7, ZINC, 5>(P, A, batch, st);
    case 8: return enc_full<8, ZINC, 5>(P, A, batch, st);
    case 9: return enc_full<9, ZINC, 5>(P, A, batch, st);
    case 10: return enc_full<10, ZINC, 5>(P, A, batch, st);
    case 11: return enc_full<11, ZINC, 5>(P, A, batch, st);
    case 12: return enc_full<12, ZINC, 5>(P, A, batch, st);
    case 13: return enc_full<13, ZINC, 5>(P, A, batch, st);
    case 14: return enc_full<14, ZINC, 5>(P, A, batch, st);
    case 15: return enc_half<14, ZINC, 5>(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_encrypt(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, int variant,
                           cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return zinc ? enc_dispatch<true>(P, A, batch, variant, st) : enc_dispatch<false>(P, A, batch, variant, st);
}

}  // namespace zn
