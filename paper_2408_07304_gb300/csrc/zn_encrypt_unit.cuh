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
// runs the same barriers but touches no global memory.  The last NTT pass
// hands its outputs over unreduced where the epilogue can absorb them: the
// Shoup product pk*u-hat takes any 64-bit input, and a sum below 32q (relaxed:
// 2q plus 2q + 2q*LOGN, the inputs being below 2q) or 8q (Harvey) is reduced
// once (reduce_sum).
// Radix-8 schedules (KM = 3) with LOGN = 1 mod 3 run the top stage in the
// generator and 3-bit passes over the rest, and stage the last pass through
// shared memory (its threads own 8 adjacent outputs each).
template <int LOGN, bool ZINC, int LOGPER, bool RELAX, int KM = 4>
__device__ __forceinline__ void encrypt_unit_q(const DevParams& P, const EncArgs& A, int i, size_t b, u64* sm, int t,
                                               bool active) {
  using S = NttShape<LOGN, LOGPER>;
  // inputs below 2q (reduce_biased), 2q per relaxed stage, 2q from the key product
  static_assert(!RELAX || 2 + 2 * LOGN + 2 <= 32, "relaxed sums must stay below 32q");
  constexpr bool TOP = KM == 3 && LOGN % 3 == 1;
  constexpr int HI = TOP ? LOGN - 1 : LOGN;
  const int L = P.L;
  const u64 q = P.q[i], mu = P.mu[i], moff = P.moff[i];
  const ulonglong2* tw = P.twp + (size_t)i * S::N;
  u64* c0 = A.out + (b * 2 * L + i) * S::N;
  u64* c1 = c0 + (size_t)L * S::N;
  const i64* me = A.me + b * S::N;
  const int8_t* sp = A.small + b * 2 * S::N;
  const u64* k0 = A.key + (size_t)i * S::N;
  const u64* k1 = k0 + (size_t)L * S::N;
  auto load_small = [&](const int8_t* src, auto tern) {
    if (!active) return;
    if constexpr (TOP) gen_i8_top<LOGN, KM, RELAX, decltype(tern)::value>(sm, t, S::T, src, q, __ldg(tw + 1));
    else gen_i8<LOGN, KM>(sm, t, S::T, src, q);
  };
  auto load_me = [&]() {
    if (!active) return;
    if constexpr (TOP) gen_i64_top<LOGN, KM, RELAX>(sm, t, S::T, me, q, mu, moff, __ldg(tw + 1));
    else gen_i64<LOGN, KM>(sm, t, S::T, me, q, mu, moff);
  };
  if constexpr (!ZINC) {
    const u64* k0s = A.keys + (size_t)i * S::N;
    const u64* k1s = k0s + (size_t)L * S::N;
    // u-hat, then the two key products (kept lazily in [0, 2q) in the output)
    load_small(sp, std::true_type{});
    auto st_u = [&](int idx, u64 uh) {
      if (!active) return;
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_u), KM, true, KM == 3>(sm, t, tw, 1, q, st_u);
    // m + e0 -> c0
    __syncthreads();
    load_me();
    auto st_0 = [&](int idx, u64 x) {
      if (active) __stcs(c0 + idx, reduce_sum<RELAX>(c0[idx] + x, q));
    };
    ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_0), KM, true, KM == 3>(sm, t, tw, 1, q, st_0);
    // e1 -> c1
    __syncthreads();
    load_small(sp + S::N, std::false_type{});
    auto st_1 = [&](int idx, u64 x) {
      if (active) __stcs(c1 + idx, reduce_sum<RELAX>(c1[idx] + x, q));
    };
    ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_1), KM, true, KM == 3>(sm, t, tw, 1, q, st_1);
  } else {
    load_me();
    auto st_0 = [&](int idx, u64 x) {
      if (active) __stcs(c0 + idx, reduce_sum<RELAX>(__ldg(k0 + idx) + x, q));
    };
    ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_0), KM, true, KM == 3>(sm, t, tw, 1, q, st_0);
    __syncthreads();
    load_small(sp, std::false_type{});
    auto st_1 = [&](int idx, u64 x) {
      if (active) __stcs(c1 + idx, reduce_sum<RELAX>(__ldg(k1 + idx) + x, q));
    };
    ntt_chain<LOGN, LOGPER, HI, RELAX, decltype(st_1), KM, true, KM == 3>(sm, t, tw, 1, q, st_1);
  }
}

// N = 2^(LOGH+1): output half h of prime i (one limb exceeds shared memory).
// Relaxed outputs start below 4q (the first stage; 6q when the generator also
// runs the half's top stage) and stay below 4q + 2q*LOGH; the sums take them
// unreduced only while that plus 2q is at most 32q (LOGH <= 13).
template <int LOGH, bool ZINC, int LOGPER, bool RELAX, int KM = 4>
__device__ __forceinline__ void encrypt_half_unit_q(const DevParams& P, const EncArgs& A, int i, int h, size_t b,
                                                    u64* sm, int t) {
  using S = NttShape<LOGH, LOGPER>;
  constexpr int N = 2 << LOGH, HALF = 1 << LOGH;
  constexpr bool RAW = !RELAX || 4 + 2 * LOGH + 2 <= 32;
  constexpr bool TOP = KM == 3 && LOGH % 3 == 1;
  constexpr int HI = TOP ? LOGH - 1 : LOGH;
  const int L = P.L;
  const u64 q = P.q[i], mu = P.mu[i], moff = P.moff[i];
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
  auto sum = [&](u64 a, u64 x) { return RAW ? reduce_sum<RELAX>(a + x, q) : reduce4(a + x, q); };
  auto load_small = [&](const int8_t* src, auto tern) {
    constexpr bool TERN = decltype(tern)::value;
    if constexpr (TOP) gen_i8_half2<LOGH, KM, RELAX, TERN>(sm, t, S::T, h, src, q, w1p, __ldg(tw + tmul), __ldg(tw + 5 - tmul));
    else gen_i8_half<LOGH, KM, TERN>(sm, t, S::T, h, src, q, w1, w1s);
  };
  auto load_me = [&]() {
    if constexpr (TOP) gen_i64_half2<LOGH, KM, RELAX>(sm, t, S::T, h, me, q, mu, moff, w1p, __ldg(tw + tmul));
    else gen_i64_half<LOGH, KM>(sm, t, S::T, h, me, q, mu, moff, w1, w1s);
  };
  if constexpr (!ZINC) {
    const u64* k0s = A.keys + (size_t)i * N + off;
    const u64* k1s = k0s + (size_t)L * N;
    load_small(sp, std::true_type{});
    auto st_u = [&](int idx, u64 uh) {
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    ntt_chain<LOGH, LOGPER, HI, RELAX, decltype(st_u), KM, true, KM == 3>(sm, t, tw, tmul, q, st_u);
    __syncthreads();
    load_me();
    auto st_0 = [&](int idx, u64 x) { c0[idx] = sum(c0[idx], x); };
    ntt_chain<LOGH, LOGPER, HI, RELAX, decltype(st_0), KM, RAW, KM == 3>(sm, t, tw, tmul, q, st_0);
    __syncthreads();
    load_small(sp + N, std::false_type{});
    auto st_1 = [&](int idx, u64 x) { c1[idx] = sum(c1[idx], x); };
    ntt_chain<LOGH, LOGPER, HI, RELAX, decltype(st_1), KM, RAW, KM == 3>(sm, t, tw, tmul, q, st_1);
  } else {
    load_me();
    auto st_0 = [&](int idx, u64 x) { c0[idx] = sum(__ldg(k0 + idx), x); };
    ntt_chain<LOGH, LOGPER, HI, RELAX, decltype(st_0), KM, RAW, KM == 3, 2>(sm, t, tw, tmul, q, st_0);
    __syncthreads();
    load_small(sp, std::false_type{});
    auto st_1 = [&](int idx, u64 x) { c1[idx] = sum(__ldg(k1 + idx), x); };
    ntt_chain<LOGH, LOGPER, HI, RELAX, decltype(st_1), KM, RAW, KM == 3, 2>(sm, t, tw, tmul, q, st_1);
  }
}

// Primes below 2^59 take the relaxed butterflies (uniform per unit); rings
// below 2^10 (tests only) always use the corrected ones.
template <int LOGN, bool ZINC, int LOGPER, int KM = 4>
__device__ __forceinline__ void encrypt_unit(const DevParams& P, const EncArgs& A, int i, size_t b, u64* sm, int t,
                                             bool active) {
  if constexpr (LOGN >= 10) {
    if (P.q[i] < kRelaxLimit) {
      encrypt_unit_q<LOGN, ZINC, LOGPER, true, KM>(P, A, i, b, sm, t, active);
      return;
    }
  }
  encrypt_unit_q<LOGN, ZINC, LOGPER, false, KM>(P, A, i, b, sm, t, active);
}

template <int LOGH, bool ZINC, int LOGPER, int KM = 4>
__device__ __forceinline__ void encrypt_half_unit(const DevParams& P, const EncArgs& A, int i, int h, size_t b,
                                                  u64* sm, int t) {
  if (P.q[i] < kRelaxLimit) encrypt_half_unit_q<LOGH, ZINC, LOGPER, true, KM>(P, A, i, h, b, sm, t);
  else encrypt_half_unit_q<LOGH, ZINC, LOGPER, false, KM>(P, A, i, h, b, sm, t);
}

}  // namespace zn


// ---------------------------------------------------- multi-polynomial units
// One block owns part h of 2^S equal output parts (S = 0: the whole limb,
// N <= 2^13; S = 1: one output half, N = 2^14) of EVERY polynomial of one
// (ciphertext, prime): u, m+e0, e1 (vanilla) or m+e1', e2' (Zinc), each in its
// own 2^LOGM-word region of shared memory, LOGM = LOGN - S.  Each register
// pass loads its group's twiddles once and applies them to all polynomials;
// the final single-stage pass keeps every polynomial's outputs in registers,
// so the epilogue combines them and writes c0, c1 once:
//   vanilla (Eq. 8):    c0 = pk0*u + (m+e0)^,  c1 = pk1*u + e1^
//   Zinc (Algorithm 1): c0' = z0 + (m+e1')^,   c1' = z1 + e2'^
// 2^(LOGM-4) threads, 16 coefficients of each polynomial per thread.
namespace zn {

template <int LOGM>
struct MpShape {
  static constexpr int M = 1 << LOGM;
  static constexpr int T = M / 16;
};

// Index bits [LO, LO+K) of every polynomial, LO >= 1.  Twiddle of stage bit
// LO+s for group element r: twp[tmul * 2^(LOGM-1-LO-s) + ghi * 2^(K-1-s) + (r >> (s+1))].
template <int LOGM, int LO, int K, int NP, bool RELAX>
__device__ __forceinline__ void mp_pass(u64* sm, int t, const ulonglong2* __restrict__ twp, int tmul, u64 q) {
  constexpr int T = MpShape<LOGM>::T, M = MpShape<LOGM>::M;
  constexpr int G = 16 >> K;
#pragma unroll 1
  for (int j = 0; j < G; ++j) {
    const int g = t + j * T;
    const int ghi = g >> LO;
    const int sb = swz<LOGM>((g & ((1 << LO) - 1)) | (ghi << (LO + K)));
    ulonglong2 w[(1 << K) - 1];      // stage s: w[2^(K-1-s) - 1 + jj], jj < 2^(K-1-s)
#pragma unroll
    for (int s = K - 1; s >= 0; --s) {
      const ulonglong2* tws = twp + (tmul << (LOGM - 1 - LO - s)) + (ghi << (K - s - 1));
#pragma unroll
      for (int jj = 0; jj < (1 << (K - 1 - s)); ++jj) w[(1 << (K - 1 - s)) - 1 + jj] = __ldg(tws + jj);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      u64* smp = sm + p * M;
      u64 v[1 << K];
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) v[r] = smp[sb ^ swz<LOGM>(r << LO)];
#pragma unroll
      for (int s = K - 1; s >= 0; --s) {
#pragma unroll
        for (int r = 0; r < (1 << K); ++r) {
          if (r & (1 << s)) continue;
          const ulonglong2 ww = w[(1 << (K - 1 - s)) - 1 + (r >> (s + 1))];
          if constexpr (RELAX) ct_bfly_relaxed(v[r], v[r + (1 << s)], ww, q);
          else ct_bfly(v[r], v[r + (1 << s)], ww, q);
        }
      }
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) smp[sb ^ swz<LOGM>(r << LO)] = v[r];
    }
  }
}

// Passes of at most 4 bits from the top down to bit 1 (bit 0 is the epilogue's).
template <int LOGM, int HI, int NP, bool RELAX>
__device__ __forceinline__ void mp_chain(u64* sm, int t, const ulonglong2* twp, int tmul, u64 q) {
  constexpr int K = (HI - 1) < 4 ? (HI - 1) : 4;
  constexpr int LO = HI - K;
  __syncthreads();
  mp_pass<LOGM, LO, K, NP, RELAX>(sm, t, twp, tmul, q);
  if constexpr (LO > 1) mp_chain<LOGM, LO, NP, RELAX>(sm, t, twp, tmul, q);
}

// Final stage (bit 0) of all NP transforms: for output pair (2g, 2g+1),
// fin(g, x0, x1) receives every polynomial's outputs, reduced to [0, q).
template <int LOGM, int NP, bool RELAX, class Fin>
__device__ __forceinline__ void mp_last(u64* sm, int t, const ulonglong2* __restrict__ twp, int tmul, u64 q,
                                        Fin& fin) {
  constexpr int T = MpShape<LOGM>::T, M = MpShape<LOGM>::M;
  __syncthreads();
#pragma unroll 1
  for (int j = 0; j < 8; ++j) {
    const int g = t + j * T;
    const int sb = swz<LOGM>(g << 1);
    const ulonglong2 w = __ldg(twp + (tmul << (LOGM - 1)) + g);
    u64 x0[NP], x1[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      u64 a = sm[p * M + sb], b = sm[p * M + (sb ^ swz<LOGM>(1))];
      if constexpr (RELAX) ct_bfly_relaxed(a, b, w, q);
      else ct_bfly(a, b, w, q);
      x0[p] = reduce_out<RELAX>(a, q);
      x1[p] = reduce_out<RELAX>(b, q);
    }
    fin(g, x0, x1);
  }
}

// Unit (prime i, ciphertext b, part h).  Output, key and companion pointers
// must be 16-byte aligned (pairs are loaded and stored as 16-byte vectors).
template <int LOGN, bool ZINC, bool RELAX>
__device__ __forceinline__ void encrypt_mp_unit_q(const DevParams& P, const EncArgs& A, int i, int h, size_t b,
                                                  u64* sm, int t) {
  constexpr int S = LOGN == 14 ? 1 : 0;
  constexpr int LOGM = LOGN - S;
  constexpr int N = 1 << LOGN, M = 1 << LOGM;
  constexpr int NP = ZINC ? 2 : 3;
  constexpr int T = MpShape<LOGM>::T;
  const int L = P.L;
  const u64 q = P.q[i], mu = P.mu[i], moff = P.moff[i];
  const ulonglong2* tw = P.twp + (size_t)i * N;
  const size_t off = (size_t)h * M;
  ulonglong2* c0 = reinterpret_cast<ulonglong2*>(A.out + (b * 2 * L + i) * N + off);
  ulonglong2* c1 = reinterpret_cast<ulonglong2*>(A.out + (b * 2 * L + L + i) * N + off);
  const i64* me = A.me + b * N;
  const int8_t* sp = A.small + b * 2 * N;
  const ulonglong2* k0 = reinterpret_cast<const ulonglong2*>(A.key + (size_t)i * N + off);
  const ulonglong2* k1 = reinterpret_cast<const ulonglong2*>(A.key + (size_t)(L + i) * N + off);
  // regions: vanilla [u, m+e0, e1], Zinc [m+e1', e2']
  if constexpr (S == 0) {
    if constexpr (!ZINC) {
      gen_i8<LOGM>(sm, t, T, sp, q);
      gen_i64<LOGM>(sm + M, t, T, me, q, mu, moff);
      gen_i8<LOGM>(sm + 2 * M, t, T, sp + N, q);
    } else {
      gen_i64<LOGM>(sm, t, T, me, q, mu, moff);
      gen_i8<LOGM>(sm + M, t, T, sp, q);
    }
  } else {
    const ulonglong2 w1 = __ldg(tw + 1);
    if constexpr (!ZINC) {
      gen_i8_half<LOGM, 4, true>(sm, t, T, h, sp, q, w1.x, w1.y);
      gen_i64_half<LOGM>(sm + M, t, T, h, me, q, mu, moff, w1.x, w1.y);
      gen_i8_half<LOGM>(sm + 2 * M, t, T, h, sp + N, q, w1.x, w1.y);
    } else {
      gen_i64_half<LOGM>(sm, t, T, h, me, q, mu, moff, w1.x, w1.y);
      gen_i8_half<LOGM>(sm + M, t, T, h, sp, q, w1.x, w1.y);
    }
  }
  const int tmul = (1 << S) + h;
  mp_chain<LOGM, LOGM, NP, RELAX>(sm, t, tw, tmul, q);
  if constexpr (!ZINC) {
    const ulonglong2* k0s = reinterpret_cast<const ulonglong2*>(A.keys + (size_t)i * N + off);
    const ulonglong2* k1s = reinterpret_cast<const ulonglong2*>(A.keys + (size_t)(L + i) * N + off);
    auto fin = [&](int g, const u64 (&x0)[NP], const u64 (&x1)[NP]) {
      const ulonglong2 a0 = __ldg(k0 + g), a0s = __ldg(k0s + g), a1 = __ldg(k1 + g), a1s = __ldg(k1s + g);
      ulonglong2 r0, r1;
      r0.x = reduce4(mul_shoup(x0[0], a0.x, a0s.x, q) + x0[1], q);    // [0, 2q) + [0, q)
      r0.y = reduce4(mul_shoup(x1[0], a0.y, a0s.y, q) + x1[1], q);
      r1.x = reduce4(mul_shoup(x0[0], a1.x, a1s.x, q) + x0[2], q);
      r1.y = reduce4(mul_shoup(x1[0], a1.y, a1s.y, q) + x1[2], q);
      c0[g] = r0;
      c1[g] = r1;
    };
    mp_last<LOGM, NP, RELAX>(sm, t, tw, tmul, q, fin);
  } else {
    auto fin = [&](int g, const u64 (&x0)[NP], const u64 (&x1)[NP]) {
      const ulonglong2 a0 = __ldg(k0 + g), a1 = __ldg(k1 + g);
      c0[g] = make_ulonglong2(reduce4(a0.x + x0[0], q), reduce4(a0.y + x1[0], q));
      c1[g] = make_ulonglong2(reduce4(a1.x + x0[1], q), reduce4(a1.y + x1[1], q));
    };
    mp_last<LOGM, NP, RELAX>(sm, t, tw, tmul, q, fin);
  }
}

template <int LOGN, bool ZINC>
__device__ __forceinline__ void encrypt_mp_unit(const DevParams& P, const EncArgs& A, int i, int h, size_t b,
                                                u64* sm, int t) {
  if (P.q[i] < kRelaxLimit) encrypt_mp_unit_q<LOGN, ZINC, true>(P, A, i, h, b, sm, t);
  else encrypt_mp_unit_q<LOGN, ZINC, false>(P, A, i, h, b, sm, t);
}

}  // namespace zn
