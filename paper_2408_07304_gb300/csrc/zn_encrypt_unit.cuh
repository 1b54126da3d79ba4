// Device-side encryption units shared by the single-ring kernels
// (zn_encrypt.cu) and the persistent mixed-ring kernel (zn_batch.cu).
//
// One unit of work is one RNS limb of one ciphertext, owned by 2^(LOGN-LOGPER)
// threads.  The unit reduces the prepared integer polynomials (sampled and
// encoded once per ciphertext by the prep kernel) mod its prime into shared
// memory, runs the negacyclic NTT (Shoup multiplication, Harvey lazy
// butterflies -- relaxed ones for primes below 2^59 --, radix-16 register
// passes), and fuses the epilogue:
//   vanilla (Eq. 8):      c0 = pk0*u + NTT(m + e0),  c1 = pk1*u + NTT(e1)
//   Zinc (Algorithm 1):   c0' = z0 + NTT(m + e1'),   c1' = z1 + NTT(e2')
#pragma once
#include "zn_kernels.h"

namespace zn {


// Full transform (N <= 2^14).  Sub-group thread t; an inactive sub-group
// runs the same barriers but touches no global memory.
template <int LOGN, bool ZINC, int LOGPER, bool RELAX>
__device__ __forceinline__ void encrypt_unit_q(const DevParams& P, const EncArgs& A, int i, size_t b, u64* sm, int t,
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
      const u64 uh = x;
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_forward_sub<LOGN, decltype(st_u), LOGPER, RELAX>(sm, t, tw, 1, q, st_u);
    // m + e0 -> c0
    __syncthreads();
    if (active) gen_i64<LOGN>(sm, t, S::T, me, q, mu);
    auto st_0 = [&](int idx, u64 x) {
      if (active) c0[idx] = reduce4(c0[idx] + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_0), LOGPER, RELAX>(sm, t, tw, 1, q, st_0);
    // e1 -> c1
    __syncthreads();
    if (active) gen_i8<LOGN>(sm, t, S::T, sp + S::N, q);
    auto st_1 = [&](int idx, u64 x) {
      if (active) c1[idx] = reduce4(c1[idx] + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_1), LOGPER, RELAX>(sm, t, tw, 1, q, st_1);
  } else {
    if (active) gen_i64<LOGN>(sm, t, S::T, me, q, mu);
    auto st_0 = [&](int idx, u64 x) {
      if (active) c0[idx] = reduce4(__ldg(k0 + idx) + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_0), LOGPER, RELAX>(sm, t, tw, 1, q, st_0);
    __syncthreads();
    if (active) gen_i8<LOGN>(sm, t, S::T, sp, q);
    auto st_1 = [&](int idx, u64 x) {
      if (active) c1[idx] = reduce4(__ldg(k1 + idx) + x, q);
    };
    ntt_forward_sub<LOGN, decltype(st_1), LOGPER, RELAX>(sm, t, tw, 1, q, st_1);
  }
}

// N = 2^(LOGH+1): output half h of prime i (one limb exceeds shared memory).
template <int LOGH, bool ZINC, int LOGPER, bool RELAX>
__device__ __forceinline__ void encrypt_half_unit_q(const DevParams& P, const EncArgs& A, int i, int h, size_t b,
                                                    u64* sm, int t) {
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
      const u64 uh = x;
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_forward_sub<LOGH, decltype(st_u), LOGPER, RELAX>(sm, t, tw, tmul, q, st_u);
    __syncthreads();
    gen_i64_half<LOGH>(sm, t, S::T, h, me, q, mu, w1, w1s);
    auto st_0 = [&](int idx, u64 x) { c0[idx] = reduce4(c0[idx] + x, q); };
    ntt_forward_sub<LOGH, decltype(st_0), LOGPER, RELAX>(sm, t, tw, tmul, q, st_0);
    __syncthreads();
    gen_i8_half<LOGH>(sm, t, S::T, h, sp + N, q, w1, w1s);
    auto st_1 = [&](int idx, u64 x) { c1[idx] = reduce4(c1[idx] + x, q); };
    ntt_forward_sub<LOGH, decltype(st_1), LOGPER, RELAX>(sm, t, tw, tmul, q, st_1);
  } else {
    gen_i64_half<LOGH>(sm, t, S::T, h, me, q, mu, w1, w1s);
    auto st_0 = [&](int idx, u64 x) { c0[idx] = reduce4(__ldg(k0 + idx) + x, q); };
    ntt_forward_sub<LOGH, decltype(st_0), LOGPER, RELAX>(sm, t, tw, tmul, q, st_0);
    __syncthreads();
    gen_i8_half<LOGH>(sm, t, S::T, h, sp, q, w1, w1s);
    auto st_1 = [&](int idx, u64 x) { c1[idx] = reduce4(__ldg(k1 + idx) + x, q); };
    ntt_forward_sub<LOGH, decltype(st_1), LOGPER, RELAX>(sm, t, tw, tmul, q, st_1);
  }
}

// Primes below 2^59 take the relaxed butterflies (uniform per unit); rings
// below 2^10 (tests only) always use the corrected ones.
template <int LOGN, bool ZINC, int LOGPER>
__device__ __forceinline__ void encrypt_unit(const DevParams& P, const EncArgs& A, int i, size_t b, u64* sm, int t,
                                             bool active) {
  if constexpr (LOGN >= 10) {
    if (P.q[i] < kRelaxLimit) {
      encrypt_unit_q<LOGN, ZINC, LOGPER, true>(P, A, i, b, sm, t, active);
      return;
    }
  }
  encrypt_unit_q<LOGN, ZINC, LOGPER, false>(P, A, i, b, sm, t, active);
}

template <int LOGH, bool ZINC, int LOGPER>
__device__ __forceinline__ void encrypt_half_unit(const DevParams& P, const EncArgs& A, int i, int h, size_t b,
                                                  u64* sm, int t) {
  if (P.q[i] < kRelaxLimit) encrypt_half_unit_q<LOGH, ZINC, LOGPER, true>(P, A, i, h, b, sm, t);
  else encrypt_half_unit_q<LOGH, ZINC, LOGPER, false>(P, A, i, h, b, sm, t);
}

}  // namespace zn
