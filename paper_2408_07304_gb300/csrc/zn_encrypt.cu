// Hot path: fused per-(prime, ciphertext) encryption for sm_103a.
//
// One unit of work is one RNS limb of one ciphertext, owned by 2^(LOGN-LOGPER)
// threads.  The unit reduces the prepared integer polynomials (sampled and
// encoded once per ciphertext by the prep kernel) mod its prime into shared
// memory, runs the negacyclic NTT (Shoup multiplication, Harvey lazy
// butterflies, radix-16 register passes), and fuses the epilogue:
//   vanilla (Eq. 8):      c0 = pk0*u + NTT(m + e0),  c1 = pk1*u + NTT(e1)
//   Zinc (Algorithm 1):   c0' = z0 + NTT(m + e1'),   c1' = z1 + NTT(e2')
//
// k_encrypt / k_encrypt_half launch one unit per block for a single ring;
// k_batch_encrypt is a persistent kernel that walks a work list of "packets"
// (same-ring units filling a 512-thread block) across rings of different
// degree, chain and mode in one launch.
#include "zn_kernels.h"

namespace zn {

// Full transform (N <= 2^14).  Sub-group thread t; an inactive sub-group
// runs the same barriers but touches no global memory.
template <int LOGN, bool ZINC, int LOGPER>
__device__ __forceinline__ void encrypt_unit(const DevParams& P, const EncArgs& A, int i, size_t b, u64* sm, int t,
                                             bool active) {
  using S = NttShape<LOGN, LOGPER>;
  const int L = P.L;
  const u64 q = P.q[i], mu = P.mu[i];
  const ulonglong2* tw = P.twp + (size_t)i * S::N;
  u64* c0 = A.out + (b * 2 * L + i) * S::N;
  u64* c1 = c0 + (size_t)L * S::N;
  const i64* me = A.me + b * S::N;
  const int8_t* sp = A.small + b * 2 * S::N;
  const u64* k0 = A.key + (size_t)i * S::N;
  const u64* k1 = k0 + (size_t)L * S::N;
  if constexpr (!ZINC) {
    const u64* k0s = A.keys + (size_t)i * S::N;
    const u64* k1s = k0s + (size_t)L * S::N;
    // u-hat, then the two key products (kept lazily in [0, 2q) in the output)
    if (active) gen_i8<LOGN>(sm, t, S::T, sp, q);
    auto st_u = [&](int idx, u64 x) {
      if (!active) return;
      const u64 uh = reduce4(x, q);
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_forward_sub<LOGN, decltype(st_u), LOGPER>(sm, t, tw, 1, q, st_u);
    // m + e0 -> c0
    __syncthreads();
    if (active) gen_i64<LOGN>(sm, t, S::T, me, q, mu);
    auto st_0 = [&](int idx, u64 x) {
      if (active) c0[idx] = reduce8(c0[idx] + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_0), LOGPER>(sm, t, tw, 1, q, st_0);
    // e1 -> c1
    __syncthreads();
    if (active) gen_i8<LOGN>(sm, t, S::T, sp + S::N, q);
    auto st_1 = [&](int idx, u64 x) {
      if (active) c1[idx] = reduce8(c1[idx] + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_1), LOGPER>(sm, t, tw, 1, q, st_1);
  } else {
    if (active) gen_i64<LOGN>(sm, t, S::T, me, q, mu);
    auto st_0 = [&](int idx, u64 x) {
      if (active) c0[idx] = reduce8(__ldg(k0 + idx) + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_0), LOGPER>(sm, t, tw, 1, q, st_0);
    __syncthreads();
    if (active) gen_i8<LOGN>(sm, t, S::T, sp, q);
    auto st_1 = [&](int idx, u64 x) {
      if (active) c1[idx] = reduce8(__ldg(k1 + idx) + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_1), LOGPER>(sm, t, tw, 1, q, st_1);
  }
}

// N = 2^(LOGH+1): output half h of prime i (one limb exceeds shared memory).
template <int LOGH, bool ZINC, int LOGPER>
__device__ __forceinline__ void encrypt_half_unit(const DevParams& P, const EncArgs& A, int i, int h, size_t b, u64* sm,
                                                  int t) {
  using S = NttShape<LOGH, LOGPER>;
  constexpr int N = 2 << LOGH, HALF = 1 << LOGH;
  const int L = P.L;
  const u64 q = P.q[i], mu = P.mu[i];
  const ulonglong2* tw = P.twp + (size_t)i * N;
  const ulonglong2 w1p = __ldg(tw + 1);
  const u64 w1 = w1p.x, w1s = w1p.y;
  const size_t off = (size_t)h * HALF;
  u64* c0 = A.out + (b * 2 * L + i) * N + off;
  u64* c1 = c0 + (size_t)L * N;
  const i64* me = A.me + b * N;
  const int8_t* sp = A.small + b * 2 * N;
  const u64* k0 = A.key + (size_t)i * N + off;
  const u64* k1 = k0 + (size_t)L * N;
  const int tmul = 2 + h;
  if constexpr (!ZINC) {
    const u64* k0s = A.keys + (size_t)i * N + off;
    const u64* k1s = k0s + (size_t)L * N;
    gen_i8_half<LOGH>(sm, t, S::T, h, sp, q, w1, w1s);
    auto st_u = [&](int idx, u64 x) {
      const u64 uh = reduce4(x, q);
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_forward_sub<LOGH, decltype(st_u), LOGPER>(sm, t, tw, tmul, q, st_u);
    __syncthreads();
    gen_i64_half<LOGH>(sm, t, S::T, h, me, q, mu, w1, w1s);
    auto st_0 = [&](int idx, u64 x) { c0[idx] = reduce8(c0[idx] + x, q); };
    ntt_forward_sub<LOGH, decltype(st_0), LOGPER>(sm, t, tw, tmul, q, st_0);
    __syncthreads();
    gen_i8_half<LOGH>(sm, t, S::T, h, sp + N, q, w1, w1s);
    auto st_1 = [&](int idx, u64 x) { c1[idx] = reduce8(c1[idx] + x, q); };
    ntt_forward_sub<LOGH, decltype(st_1), LOGPER>(sm, t, tw, tmul, q, st_1);
  } else {
    gen_i64_half<LOGH>(sm, t, S::T, h, me, q, mu, w1, w1s);
    auto st_0 = [&](int idx, u64 x) { c0[idx] = reduce8(__ldg(k0 + idx) + x, q); };
    ntt_forward_sub<LOGH, decltype(st_0), LOGPER>(sm, t, tw, tmul, q, st_0);
    __syncthreads();
    gen_i8_half<LOGH>(sm, t, S::T, h, sp, q, w1, w1s);
    auto st_1 = [&](int idx, u64 x) { c1[idx] = reduce8(__ldg(k1 + idx) + x, q); };
    ntt_forward_sub<LOGH, decltype(st_1), LOGPER>(sm, t, tw, tmul, q, st_1);
  }
}

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

// variant 0: 32 elements per thread; variant 1: 16 elements per thread (rings >= 2^12)
template <bool ZINC>
static cudaError_t enc_dispatch(const DevParams& P, const EncArgs& A_in, uint32_t batch, int variant,
                                cudaStream_t st) {
  const bool v1 = (variant & 1) != 0;
  EncArgs A = A_in;
  A.swap = (variant >> 1) & 1;
  switch (P.log_n) {
    case 4: return enc_full<4, ZINC, 5>(P, A, batch, st);
    case 5: return enc_full<5, ZINC, 5>(P, A, batch, st);
    case 6: return enc_full<6, ZINC, 5>(P, A, batch, st);
    case 7: return enc_full<7, ZINC, 5>(P, A, batch, st);
    case 8: return enc_full<8, ZINC, 5>(P, A, batch, st);
    case 9: return enc_full<9, ZINC, 5>(P, A, batch, st);
    case 10: return enc_full<10, ZINC, 5>(P, A, batch, st);
    case 11: return enc_full<11, ZINC, 5>(P, A, batch, st);
    case 12: return v1 ? enc_full<12, ZINC, 4>(P, A, batch, st) : enc_full<12, ZINC, 5>(P, A, batch, st);
    case 13: return v1 ? enc_full<13, ZINC, 4>(P, A, batch, st) : enc_full<13, ZINC, 5>(P, A, batch, st);
    case 14: return v1 ? enc_full<14, ZINC, 4>(P, A, batch, st) : enc_full<14, ZINC, 5>(P, A, batch, st);
    case 15: return v1 ? enc_half<14, ZINC, 4>(P, A, batch, st) : enc_half<14, ZINC, 5>(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_encrypt(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, int variant,
                           cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return zinc ? enc_dispatch<true>(P, A, batch, variant, st) : enc_dispatch<false>(P, A, batch, variant, st);
}

// -------------------------------------------------- mixed rings, persistent

// Packet: `count` units of one job -- ciphertexts b0 .. b0+count-1 at prime
// `prime` (half `half` for N = 2^15) -- processed together by one 512-thread
// block, 2^(LOGN-5) threads and 2^LOGN shared words per unit.
template <int LOGN, bool ZINC>
__device__ __forceinline__ void batch_full(const JobDesc& J, const EncPacket& pk, u64* sm) {
  using S = NttShape<LOGN, 5>;
  const int g = threadIdx.x / S::T, t = threadIdx.x % S::T;
  encrypt_unit<LOGN, ZINC, 5>(J.P, J.E, pk.prime, (size_t)pk.b0 + g, sm + (size_t)g * S::N, t, g < (int)pk.count);
}

template <bool ZINC>
__device__ __forceinline__ void batch_packet(const JobDesc& J, const EncPacket& pk, u64* sm) {
  switch (J.P.log_n) {
    case 10: batch_full<10, ZINC>(J, pk, sm); break;
    case 11: batch_full<11, ZINC>(J, pk, sm); break;
    case 12: batch_full<12, ZINC>(J, pk, sm); break;
    case 13: batch_full<13, ZINC>(J, pk, sm); break;
    case 14: batch_full<14, ZINC>(J, pk, sm); break;
    case 15: encrypt_half_unit<14, ZINC, 5>(J.P, J.E, pk.prime, pk.half, pk.b0, sm, threadIdx.x); break;
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
