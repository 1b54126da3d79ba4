// Hot path, multi-polynomial form (2^10 <= N <= 2^14): one block holds all
// polynomials of one limb -- of one output half of it for N = 2^14 -- and
// shares each twiddle load between them.  The unit code lives in
// zn_encrypt_unit.cuh.
#include "zn_encrypt_unit.cuh"

namespace zn {

// grid (L << S, B), or (B, L << S) when A.swap; unit (i << S) + h produces
// output part h of prime i (S = 1 for N = 2^14, else 0)
template <int LOGN, bool ZINC>
__global__ void __launch_bounds__(MpShape<LOGN - (LOGN == 14)>::T) k_encrypt_mp(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  constexpr int S = LOGN == 14 ? 1 : 0;
  const int u = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  encrypt_mp_unit<LOGN, ZINC>(P, A, u >> S, u & ((1 << S) - 1), b, sm, threadIdx.x);
}

template <int LOGN, bool ZINC>
static cudaError_t enc_mp(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  constexpr int S = LOGN == 14 ? 1 : 0;
  using M = MpShape<LOGN - S>;
  const size_t smem = sizeof(u64) * M::M * (ZINC ? 2 : 3);
  auto kern = k_encrypt_mp<LOGN, ZINC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned units = (unsigned)P.L << S;
  const dim3 grid = A.swap ? dim3(batch, units) : dim3(units, batch);
  kern<<<grid, M::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

template <bool ZINC>
static cudaError_t enc_mp_dispatch(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  switch (P.log_n) {
    case 10: return enc_mp<10, ZINC>(P, A, batch, st);
    case 11: return enc_mp<11, ZINC>(P, A, batch, st);
    case 12: return enc_mp<12, ZINC>(P, A, batch, st);
    case 13: return enc_mp<13, ZINC>(P, A, batch, st);
    case 14: return enc_mp<14, ZINC>(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_encrypt_mp(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return zinc ? enc_mp_dispatch<true>(P, A, batch, st) : enc_mp_dispatch<false>(P, A, batch, st);
}

}  // namespace zn
