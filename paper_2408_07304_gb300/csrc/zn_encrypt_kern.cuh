// Per-polynomial encryption kernels and their launchers, shared by the
// translation units that instantiate them (zn_encrypt.cu: uncapped registers;
// zn_encrypt_occ.cu and zn_encrypt_occ3.cu: register-capped shapes with two
// or three resident blocks per SM).
#pragma once
#include "zn_encrypt_unit.cuh"

namespace zn {

// grid (L, B), or (B, L) when A.swap
// MINB: resident blocks per SM the register allocation must allow; KM: bits
// per register pass (radix 2^KM).
template <int LOGN, bool ZINC, int LOGPER, int MINB = 1, int KM = 4>
__global__ void __launch_bounds__(NttShape<LOGN, LOGPER>::T, MINB) k_encrypt(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  const int i = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  encrypt_unit<LOGN, ZINC, LOGPER, KM>(P, A, i, b, sm, threadIdx.x, true);
}

// grid (2L, B), or (B, 2L) when A.swap; unit 2i + h produces output half h of prime i
template <int LOGH, bool ZINC, int LOGPER, int MINB = 1, int KM = 4>
__global__ void __launch_bounds__(NttShape<LOGH, LOGPER>::T, MINB) k_encrypt_half(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  const int u = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  encrypt_half_unit<LOGH, ZINC, LOGPER, KM>(P, A, u >> 1, u & 1, b, sm, threadIdx.x);
}

template <int LOGN, bool ZINC, int LOGPER, int MINB = 1, int KM = 4>
static cudaError_t enc_full(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGN, LOGPER>;
  const size_t smem = sizeof(u64) * S::N;
  auto kern = k_encrypt<LOGN, ZINC, LOGPER, MINB, KM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid = A.swap ? dim3(batch, P.L) : dim3(P.L, batch);
  kern<<<grid, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

template <int LOGH, bool ZINC, int LOGPER, int MINB = 1, int KM = 4>
static cudaError_t enc_half(const DevParams& P, const EncArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGH, LOGPER>;
  const size_t smem = sizeof(u64) * S::N;
  auto kern = k_encrypt_half<LOGH, ZINC, LOGPER, MINB, KM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid = A.swap ? dim3(batch, 2 * P.L) : dim3(2 * P.L, batch);
  kern<<<grid, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

static inline bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace zn
