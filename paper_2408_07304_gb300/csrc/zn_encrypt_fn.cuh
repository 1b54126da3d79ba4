// Encryption units driven by value functors, shared by the encryption forms
// whose inputs are not the plain (m + e, small) integers of the CKKS path:
// the modulus-switched vanilla encryption (zn_encrypt_ms.cu) and the BFV / BGV
// encryptions and their Zinc forms (zn_encrypt_int.cu).
//
// A unit is one RNS limb of one ciphertext (N <= 2^13 here; the cluster
// units at 2^14 and 2^15, zn_pair.cuh and zn_quarter.cuh, take the same
// functors).  Its two transform inputs come from functors v0(k), v1(k)
// returning the residue of coefficient k in [0, 2q):
//   vanilla shape:  c0 = k0 * NTT(u) + NTT(v0),   c1 = k1 * NTT(u) + NTT(v1)
//   Zinc shape:     c0 = z0 + NTT(v0),            c1 = z1 + NTT(v1)
// with the schedules of the plain units (zn_encrypt_unit.cuh): radix 2^KM,
// top stage in the generator for radix-8 chains with LOGN = 1 mod 3, staged
// last pass for radix 8, unreduced transform outputs absorbed by the sums.
#pragma once
#include "zn_kernels.h"

namespace zn {

// --------------------------------------------------- generators from values
// As gen_i64 and its variants, for a coefficient given by v(k) in [0, 2q).
template <int LOGN, int KM, class V>
__device__ __forceinline__ void gen_val(u64* sm, int t, int nt, V& v) {
  for (int k = t; k < (1 << LOGN); k += nt) sm[swz<LOGN, KM>(k)] = v(k);
}

template <int LOGN, int KM, bool RELAX, class V>
__device__ __forceinline__ void gen_val_top(u64* sm, int t, int nt, V& v, u64 q, ulonglong2 w1) {
  constexpr int H = (1 << LOGN) / 2;
  for (int k = t; k < H; k += nt) {
    u64 x = v(k), y = v(k + H);
    bfly<RELAX>(x, y, w1, q);
    sm[swz<LOGN, KM>(k)] = x;
    sm[swz<LOGN, KM>(k + H)] = y;
  }
}

// The CKKS transform input m + e, stored by the prep kernel with the offset
// 2^62: [0, 2q) after one Barrett step.
struct MeVal {
  const i64* me;
  u64 q, mu, moff;
  __device__ __forceinline__ u64 operator()(int k) const { return reduce_biased((u64)__ldg(me + k), q, mu, moff); }
};

// Output limb (or half) of a unit and its key operands.
struct FnLimb {
  u64* c0;
  u64* c1;
  const u64* k0;    // vanilla: key (NTT form); Zinc: cached zero
  const u64* k1;
  const u64* k0s;   // vanilla: Shoup companions of k0, k1
  const u64* k1s;
  const int8_t* u;  // vanilla: u, int8 [N]
};

// Write a finished ciphertext word: plain, or (STREAM) with a streaming
// (evict-first) store, which leaves L2 to the words the epilogues still
// read back.
template <bool STREAM>
__device__ __forceinline__ void put_ct(u64* p, u64 v) {
  if constexpr (STREAM) __stcs(p, v);
  else *p = v;
}

// Full transform (N = 2^LOGN <= 2^14).
template <int LOGN, int LOGPER, bool RELAX, int KM, bool ZINC, bool STREAM, class V0, class V1>
__device__ __forceinline__ void fn_unit_q(const ulonglong2* tw, u64 q, const FnLimb& o, const V0& v0, const V1& v1,
                                          u64* sm, int t) {
  using S = NttShape<LOGN, LOGPER>;
  // inputs below 2q, 2q per relaxed stage, 2q from the key product
  static_assert(!RELAX || 2 + 2 * LOGN + 2 <= 32, "relaxed sums must stay below 32q");
  constexpr bool TOP = KM == 3 && LOGN % 3 == 1;
  constexpr int HI = TOP ? LOGN - 1 : LOGN;
  u64* c0 = o.c0;
  u64* c1 = o.c1;
  const u64* k0 = o.k0;
  const u64* k1 = o.k1;
  if constexpr (!ZINC) {
    const u64* k0s = o.k0s;
    const u64* k1s = o.k1s;
    if constexpr (TOP) gen_i8_top<LOGN, KM, RELAX, true>(sm, t, S::T, o.u, q, __ldg(tw + 1));
    else gen_i8<LOGN, KM>(sm, t, S::T, o.u, q);
    auto st_u = [&](int idx, u64 uh) {
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_u), KM, true, KM == 3>(sm, t, tw, 1, q, st_u);
    __syncthreads();
  }
  if constexpr (TOP) gen_val_top<LOGN, KM, RELAX>(sm, t, S::T, v0, q, __ldg(tw + 1));
  else gen_val<LOGN, KM>(sm, t, S::T, v0);
  auto st_0 = [&](int idx, u64 x) { put_ct<STREAM>(c0 + idx, reduce_sum<RELAX>((ZINC ? __ldg(k0 + idx) : c0[idx]) + x, q)); };
  ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_0), KM, true, KM == 3>(sm, t, tw, 1, q, st_0);
  __syncthreads();
  if constexpr (TOP) gen_val_top<LOGN, KM, RELAX>(sm, t, S::T, v1, q, __ldg(tw + 1));
  else gen_val<LOGN, KM>(sm, t, S::T, v1);
  auto st_1 = [&](int idx, u64 x) { put_ct<STREAM>(c1 + idx, reduce_sum<RELAX>((ZINC ? __ldg(k1 + idx) : c1[idx]) + x, q)); };
  ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_1), KM, true, KM == 3>(sm, t, tw, 1, q, st_1);
}


}  // namespace zn
