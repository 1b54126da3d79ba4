// Hot path, one ring per launch: k_encrypt (N <= 2^14, one block per prime
// and ciphertext) and k_encrypt_half (N = 2^15, two blocks per prime and
// ciphertext).  The unit code lives in zn_encrypt_unit.cuh.
#include "zn_encrypt_unit.cuh"

namespace zn {

// ------------------------------------------------------- one ring per launch

// grid (L, B), or (B, L) when A.swap
template <int LOGN, bool ZINC, int LOGPER>
__global__ void __launch_bounds__(NttShape<LOGN, LOGPER>::T) k_encrypt(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  const int i = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  encrypt_unit<LOGN, ZINC, LOGPER>(P, A, i, b, sm, threadIdx.x, true);
}

// grid (2L, B), or (B, 2L) when A.swap; unit 2i + h produces output half h of prime i
template <int LOGH, bool ZINC, int LOGPER>
__global__ void __launch_bounds__(NttShape<LOGH, LOGPER>::T) k_encrypt_half(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  const int u = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  encrypt_half_unit<LOGH, ZINC, LOGPER>(P, A, u >> 1, u & 1, b, sm, threadIdx.x);
}

template <int LOGN, bool ZINC, int LOGPER>
static cudaError_t enc_full(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGN, LOGPER>;
  const size_t smem = sizeof(u64) * S::N;
  auto kern = k_encrypt<LOGN, ZINC, LOGPER>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid = A.swap ? dim3(batch, P.L) : dim3(P.L, batch);
  kern<<<grid, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

template <int LOGH, bool ZINC, int LOGPER>
static cudaError_t enc_half(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGH, LOGPER>;
  const size_t smem = sizeof(u64) * S::N;
  auto kern = k_encrypt_half<LOGH, ZINC, LOGPER>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid = A.swap ? dim3(batch, 2 * P.L) : dim3(2 * P.L, batch);
  kern<<<grid, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

// variant: grid order (0 prime-major, 1 ciphertext-major)
template <bool ZINC>
static cudaError_t enc_dispatch(const DevParams& P, const EncArgs& A_in, uint32_t batch, int variant,
                                cudaStream_t st) {
  EncArgs A = A_in;
  A.swap = variant & 1;
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
