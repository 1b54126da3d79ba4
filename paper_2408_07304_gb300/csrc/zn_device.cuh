// Device-side building blocks for the sm_103a encryption path:
//   * 64-bit modular arithmetic (Shoup multiplication by a precomputed
//     constant, Barrett reduction of signed integers, Harvey lazy butterflies);
//   * Philox4x32-10 and the three samplers (R_2, chi, R_q);
//   * a shared-memory-staged negacyclic NTT with radix-16 register passes;
//   * the fixed-point (Q62, exact 128-bit products) radix-2 FFT of the CKKS
//     encoder and the FP64 one of the decoder.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace zn {

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

constexpr int kMaxL = 16;
constexpr int kCdt = 38;
constexpr int kBound = 19;

// Everything a kernel needs about one parameter set; passed by value.
struct DevParams {
  int log_n, L, log2_delta, pad;
  u64 q[kMaxL];
  u64 mu[kMaxL];             // floor(2^64 / q): Barrett reduction
  u64 moff[kMaxL];           // -2^62 mod q: removes the offset of the prepared int64 polynomials
  u64 ninv[kMaxL];           // N^-1 mod q
  u64 ninvs[kMaxL];          // its Shoup companion
  u64 q0inv_mod_q1;          // CRT (decode)
  u64 cdt[kCdt];             // chi thresholds
  const ulonglong2* twp;     // [L][N] (psi^brv(k), Shoup companion) pairs
  const u64* itw;            // [L][N] psi^-brv(k)
  const u64* itws;
  const double* etw;         // [2][N] decoder twiddles (FP64): re, then im
  const longlong2* etq;      // [N] encoder twiddles (C[k], -S[k]), Q62
  const int* slot_of_t;      // [N/2] slot j with (5^j mod 2N - 1)/4 = t
  const int* pos_of_slot;    // [N/2] slot j's place in the encoder FFT input (< N/4: re, else im)
  unsigned* status;          // device status word (bit 0: encode overflow)
};

enum : unsigned { kStatusOverflow = 1u, kStatusTimeout = 2u, kStatusRange = 4u };

// ------------------------------------------------------------ modular math

// x*w mod q up to one q: result in [0, 2q) for any x < 2^64 (w < q, wp = floor(w 2^64 / q)).
__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q) {
  u64 h = __umul64hi(x, wp);
  return x * w - h * q;
}

// [0, 4q) -> [0, q)
__device__ __forceinline__ u64 reduce4(u64 x, u64 q) {
  if (x >= 2 * q) x -= 2 * q;
  if (x >= q) x -= q;
  return x;
}

// [0, 8q) -> [0, q)
__device__ __forceinline__ u64 reduce8(u64 x, u64 q) {
  if (x >= 4 * q) x -= 4 * q;
  return reduce4(x, q);
}

// signed 64-bit integer -> residue in [0, q)
__device__ __forceinline__ u64 reduce_signed(i64 x, u64 q, u64 mu) {
  u64 a = x < 0 ? (u64)0 - (u64)x : (u64)x;
  u64 r = a - __umul64hi(a, mu) * q;       // [0, 2q)
  if (r >= q) r -= q;
  return (x < 0 && r) ? q - r : r;
}

// x = v + 2^62 (stored unsigned) for a signed v with |v| < 2^62 + 2^5 ->
// v mod q in [0, 2q): one Barrett step leaves x mod q in [0, 2q), moff =
// -2^62 mod q removes the offset.
__device__ __forceinline__ u64 reduce_biased(u64 x, u64 q, u64 mu, u64 moff) {
  const u64 r = x - __umul64hi(x, mu) * q + moff;   // [0, 3q)
  return r >= 2 * q ? r - q : r;
}

// small signed integer (|v| < q) -> residue
__device__ __forceinline__ u64 small_res(int v, u64 q) {
  return v < 0 ? q - (u64)(-(i64)v) : (u64)v;
}

// v w mod q for a ternary v (v in {-1, 0, 1}) and w in [0, q): a selection,
// in [0, q].
__device__ __forceinline__ u64 mul_tern(int v, u64 w, u64 q) {
  return v == 0 ? 0ull : v > 0 ? w : q - w;
}

// v w mod q in [0, 2q) for a small signed v (|v| < 2^31) and w with Shoup
// companion ws: Shoup's quotient floor(|v| ws / 2^64) and the low word of
// |v| w built from 32 x 64-bit products instead of 64 x 64-bit ones (the same
// quotient as mul_shoup, so |v| w - quotient q lies in [0, 2q)); a negative v
// takes 2q minus that (nonzero: the prime q divides neither |v| nor w).
__device__ __forceinline__ u64 mul_small(int v, u64 w, u64 ws, u64 q) {
  const unsigned a = (unsigned)(v < 0 ? -v : v);
  const u64 lo = (u64)(unsigned)ws * a;
  const unsigned qh = (unsigned)(((u64)(unsigned)(ws >> 32) * a + (lo >> 32)) >> 32);
  const u64 aw = (u64)(unsigned)w * a + (((u64)(unsigned)(w >> 32) * a) << 32);
  const u64 r = aw - ((u64)(unsigned)q * qh + (((u64)(unsigned)(q >> 32) * qh) << 32));
  return v < 0 ? 2 * q - r : r;
}

// general a*b mod q (slow path: keygen and imports only)
__device__ __forceinline__ u64 mulmod_slow(u64 a, u64 b, u64 q) {
  return (u64)(((u128)a * b) % q);
}
__device__ __forceinline__ u64 shoup_of(u64 w, u64 q) {
  return (u64)(((u128)w << 64) / q);
}

// Harvey forward (Cooley-Tukey) butterfly; inputs and outputs in [0, 4q).
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, u64 w, u64 wp, u64 q) {
  u64 a = x >= 2 * q ? x - 2 * q : x;
  u64 t = mul_shoup(y, w, wp, q);
  x = a + t;
  y = a - t + 2 * q;
}
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, ulonglong2 w, u64 q) { ct_bfly(x, y, w.x, w.y, q); }

// Relaxed forward butterfly for q < 2^59: no correction step.  If both
// inputs are below B, both outputs are below B + 2q; a transform starting
// from [0, 4q) stays below 4q + 14 * 2q = 32q < 2^64 over 14 stages.
constexpr u64 kRelaxLimit = 1ull << 59;
__device__ __forceinline__ void ct_bfly_relaxed(u64& x, u64& y, ulonglong2 w, u64 q) {
  const u64 t = mul_shoup(y, w.x, w.y, q);   // [0, 2q)
  const u64 a = x;
  x = a + t;
  y = a - t + 2 * q;
}

// A sum below 32q (relaxed, q < 2^59) or below 8q (Harvey) -> [0, q).
template <bool RELAX>
__device__ __forceinline__ u64 reduce_sum(u64 x, u64 q) {
  if constexpr (RELAX) {
    if (x >= 16 * q) x -= 16 * q;
    if (x >= 8 * q) x -= 8 * q;
  }
  return reduce8(x, q);
}

// Output of a transform -> [0, q): Harvey range [0, 4q), relaxed range [0, 32q).
template <bool RELAX>
__device__ __forceinline__ u64 reduce_out(u64 x, u64 q) {
  if constexpr (RELAX) {
    if (x >= 16 * q) x -= 16 * q;
    if (x >= 8 * q) x -= 8 * q;
    if (x >= 4 * q) x -= 4 * q;
  }
  return reduce4(x, q);
}

// ------------------------------------------------------------------ Philox

__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// counter = (block, domain<<24 | poly<<16 | prime, lo32 ct, hi32 ct), key = seed
__device__ __forceinline__ uint4 zn_rand(u64 seed, unsigned block, unsigned tag, u64 ct) {
  return philox10(make_uint4(block, tag, (unsigned)ct, (unsigned)(ct >> 32)),
                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}
__device__ __forceinline__ unsigned rand_tag(unsigned domain, unsigned poly, unsigned prime) {
  return (domain << 24) | (poly << 16) | prime;
}

// R_2: floor(3 w / 2^32) - 1
__device__ __forceinline__ int ternary_of(unsigned w) {
  return (int)(((u64)w * 3ull) >> 32) - 1;
}

// chi: -19 + #{j : U >= T_j}
__device__ __forceinline__ int cdt_of(unsigned lo, unsigned hi, const u64* cdt) {
  u64 u = ((u64)hi << 32) | lo;
  int c = 0;
#pragma unroll
  for (int j = 0; j < kCdt; ++j) c += (u >= cdt[j]) ? 1 : 0;
  return c - kBound;
}

// The chi thresholds with a bucket index over the top 8 bits of U, staged in
// shared memory: bucket x covers U in [x 2^56, (x + 1) 2^56); b[x] holds
// lo = #{j : T_j <= x 2^56} and hi = #{j : T_j <= (x + 1) 2^56 - 1}.  The
// thresholds are sorted, so for U in bucket x the count #{j : T_j <= U} is
// lo plus the thresholds T_lo.. T_(hi-1) not above U: one shared-memory load
// when lo = hi (most buckets hold no threshold), a short scan otherwise.
struct CdtTab {
  u64 t[kCdt];
  uint16_t b[256];
};

// All threads of the block; ends with a barrier.
__device__ __forceinline__ void stage_cdt_tab(const u64* cdt, CdtTab& T) {
  for (int j = threadIdx.x; j < kCdt; j += blockDim.x) T.t[j] = cdt[j];
  for (int x = threadIdx.x; x < 256; x += blockDim.x) {
    const u64 a = (u64)x << 56, e = a + ((1ull << 56) - 1);
    int lo = 0, hi = 0;
    for (int j = 0; j < kCdt; ++j) {
      lo += cdt[j] <= a ? 1 : 0;
      hi += cdt[j] <= e ? 1 : 0;
    }
    T.b[x] = (uint16_t)(lo | (hi << 8));
  }
  __syncthreads();
}

// chi: -19 + #{j : U >= T_j} by the bucket index (the same count as cdt_of).
__device__ __forceinline__ int cdt_lookup(unsigned lo, unsigned hi, const CdtTab& T) {
  const u64 u = ((u64)hi << 32) | lo;
  const unsigned e = T.b[hi >> 24];
  int pos = (int)(e & 0xffu);
  const int top = (int)(e >> 8);
  while (pos < top && u >= T.t[pos]) ++pos;     // at most kCdt steps
  return pos - kBound;
}

// R_q: floor(W q / 2^128), W = w3:w2:w1:w0
__device__ __forceinline__ u64 uniform_of(uint4 w, u64 q) {
  u64 lo = ((u64)w.y << 32) | w.x, hi = ((u64)w.w << 32) | w.z;
  u64 a = __umul64hi(lo, q);
  u64 plo = hi * q, phi = __umul64hi(hi, q);
  u64 s = plo + a;
  return phi + (s < a ? 1ull : 0ull);
}

// ------------------------------------------------------------------ NTT

// LOGPER: log2 of the elements each thread owns (5: 32 elements, 2^(LOGN-5)
// threads; 4: 16 elements, twice the threads, half the registers each).
template <int LOGN, int LOGPER = 5>
struct NttShape {
  static constexpr int N = 1 << LOGN;
  static constexpr int LOGT = LOGN >= LOGPER ? LOGN - LOGPER : 0;
  static constexpr int T = 1 << LOGT;                 // threads per transform
  static constexpr int PER = N / T;                   // elements per thread
  static constexpr int KMAX = 4;                      // default butterfly stages per register pass
  // shared-memory swizzle i ^ ((i >> SA) & 15) ^ ((i >> SB) & 15): a bijection that
  // keeps every phase's 64-bit accesses (and the generators' consecutive
  // writes) free of bank conflicts; parameters found by exhaustive check per N
  static constexpr int SA = LOGN <= 9 ? 2 : LOGN == 10 ? 3 : LOGN == 11 ? 4 : LOGN == 12 ? 2 : LOGN == 13 ? 2
                          : LOGN == 14 ? 3 : 4;
  static constexpr int SB = LOGN <= 7 ? SA : LOGN == 8 ? 3 : LOGN == 9 ? 5 : LOGN == 10 ? 4 : LOGN == 11 ? 4
                          : LOGN == 12 ? 4 : LOGN == 13 ? 5 : 4;
};

// KM = 4: the layout of radix-16 pass schedules (parameters above); KM = 3:
// the layout of radix-8 schedules (passes of 3 bits, one of 4 absorbing a
// remainder of 1), i ^ ((i >> 1) & 15) ^ ((i >> 3) & 15), conflict-free for
// those schedules at 2^10 <= N <= 2^13 by the same exhaustive check.
template <int LOGN, int KM = 4>
__host__ __device__ constexpr int swz(int i) {
  using S = NttShape<LOGN>;
  if constexpr (KM == 3) return i ^ ((i >> 1) & 15) ^ ((i >> 3) & 15);
  return S::SA == S::SB ? (i ^ ((i >> S::SA) & 15)) : (i ^ ((i >> S::SA) & 15) ^ ((i >> S::SB) & 15));
}
// The swizzle is linear over GF(2): swz(a ^ b) = swz(a) ^ swz(b).  A group's
// slots are swz(base) ^ swz(r << LO), the second term a compile-time constant.

// One pass over index bits [LO, LO+K): each thread takes its groups of 2^K
// elements (one group at a time, in registers), runs K butterfly stages and
// writes the group back to the same shared-memory slots -- or, in the last
// pass (LO == 0), hands every output to store(idx, x): x reduced to [0, q),
// or (RAW) as the butterflies left it, below the input bound plus 2q per
// stage (relaxed) or below 4q (Harvey).  The twiddle of stage bit b for index
// idx is tw[tmul * 2^(LOGN-1-b) + (idx >> (b+1))]; tmul = 1 for a full
// transform, 2 + h for half h of a transform of twice the size.  KM selects
// the shared-memory layout (swz).
template <int LOGN, int LOGPER, int LO, int K, bool RELAX, class Store, int KM = 4, bool RAW = false,
          bool STAGED = false>
__device__ __forceinline__ void ntt_pass(u64* sm, int t, const ulonglong2* __restrict__ twp, int tmul, u64 q,
                                         Store& store) {
  using S = NttShape<LOGN, LOGPER>;
  constexpr int G = S::PER >> K;
#pragma unroll 1
  for (int j = 0; j < G; ++j) {
    const int g = t + j * S::T;
    const int ghi = g >> LO;
    const int base = (g & ((1 << LO) - 1)) | (ghi << (LO + K));
    const int sb = swz<LOGN, KM>(base);
    u64 v[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) v[r] = sm[sb ^ swz<LOGN, KM>(r << LO)];
#pragma unroll
    for (int s = K - 1; s >= 0; --s) {
      const ulonglong2* tws = twp + (tmul << (LOGN - 1 - LO - s)) + (ghi << (K - s - 1));
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) {
        if (r & (1 << s)) continue;
        if constexpr (RELAX) ct_bfly_relaxed(v[r], v[r + (1 << s)], __ldg(tws + (r >> (s + 1))), q);
        else ct_bfly(v[r], v[r + (1 << s)], __ldg(tws + (r >> (s + 1))), q);
      }
    }
    if constexpr (LO == 0 && !STAGED) {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) {
        if constexpr (RAW) store(base | r, v[r]);
        else store(base | r, reduce_out<RELAX>(v[r], q));
      }
    } else {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) sm[sb ^ swz<LOGN, KM>(r << LO)] = v[r];
    }
  }
}

// Passes of KM bits (radix 2^KM) over index bits [0, HI), from the top down
// (HI < LOGN when a generator has already run the stages above HI).
// STAGED: the last pass writes back to shared memory like the others and the
// outputs are handed to store() in natural index order (consecutive lanes,
// consecutive indices), which keeps the epilogue's global accesses coalesced
// when the last pass owns several adjacent outputs per thread; EU is that
// loop's unroll factor (a register-pressure knob: 4 keeps the vanilla units
// spill-free at 80 registers, 2 the Zinc ones).
template <int LOGN, int LOGPER, int HI, bool RELAX, class Store, int KM = NttShape<LOGN>::KMAX, bool RAW = false,
          bool STAGED = false, int EU = 4>
__device__ __forceinline__ void ntt_chain(u64* sm, int t, const ulonglong2* twp, int tmul, u64 q, Store& store) {
  constexpr int K = HI < KM ? HI : KM;
  constexpr int LO = HI - K;
  __syncthreads();
  ntt_pass<LOGN, LOGPER, LO, K, RELAX, Store, KM, RAW, STAGED>(sm, t, twp, tmul, q, store);
  if constexpr (LO > 0) {
    ntt_chain<LOGN, LOGPER, LO, RELAX, Store, KM, RAW, STAGED, EU>(sm, t, twp, tmul, q, store);
  } else if constexpr (STAGED) {
    __syncthreads();
#pragma unroll EU
    for (int idx = t; idx < (1 << LOGN); idx += NttShape<LOGN, LOGPER>::T) {
      const u64 x = sm[swz<LOGN, KM>(idx)];
      if constexpr (RAW) store(idx, x);
      else store(idx, reduce_out<RELAX>(x, q));
    }
  }
}

// Forward negacyclic NTT of one length-2^LOGN polynomial by the block's
// 2^LOGT threads.  On entry sm[swz(k)] holds coefficient k in [0, 4q) (written
// by one of the generators below; the call begins with a barrier).  store(idx,
// x) is called once per output index with x in [0, q), x = ahat[idx].
// RELAX (only for q < 2^59) drops the butterflies' correction steps.  The
// shared buffer may be reused after a barrier.
template <int LOGN, class Store, int LOGPER = 5, bool RELAX = false>
__device__ __forceinline__ void ntt_forward(u64* sm, const ulonglong2* twp, int tmul, u64 q, Store& store) {
  ntt_chain<LOGN, LOGPER, LOGN, RELAX, Store>(sm, threadIdx.x, twp, tmul, q, store);
}

// The same transform run by a sub-group of the block: thread t of the 2^LOGT
// threads that own this polynomial (several sub-groups may share one block;
// all of them must execute the same sequence of transforms, because the
// passes are separated by block-wide barriers).
template <int LOGN, class Store, int LOGPER = 5, bool RELAX = false, int KM = NttShape<LOGN>::KMAX,
          bool RAW = false>
__device__ __forceinline__ void ntt_forward_sub(u64* sm, int t, const ulonglong2* twp, int tmul, u64 q,
                                                Store& store) {
  ntt_chain<LOGN, LOGPER, LOGN, RELAX, Store, KM, RAW>(sm, t, twp, tmul, q, store);
}

// ------------------------------------------------------------- generators
// Each generator writes one polynomial into the swizzled shared buffer with
// plain block-strided loops (one Philox call per loop trip).  Callers must
// place a barrier between the previous transform's last shared-memory read
// and the generator (ntt_forward's last phase reads shared memory).

// R_2 polynomial: coefficient k comes from block k mod N/4, word k div N/4.
template <int LOGN>
__device__ __forceinline__ void gen_ternary(u64* sm, u64 seed, unsigned tag, u64 ct, u64 q) {
  constexpr int Q4 = (1 << LOGN) / 4;
  for (int blk = threadIdx.x; blk < Q4; blk += blockDim.x) {
    const uint4 w = zn_rand(seed, (unsigned)blk, tag, ct);
    sm[swz<LOGN>(blk)] = small_res(ternary_of(w.x), q);
    sm[swz<LOGN>(blk + Q4)] = small_res(ternary_of(w.y), q);
    sm[swz<LOGN>(blk + 2 * Q4)] = small_res(ternary_of(w.z), q);
    sm[swz<LOGN>(blk + 3 * Q4)] = small_res(ternary_of(w.w), q);
  }
}

// chi polynomial (+ optional message m): coefficient k from block k mod N/2,
// words (0,1) for k < N/2 and (2,3) for k >= N/2.
template <int LOGN>
__device__ __forceinline__ void gen_gauss(u64* sm, u64 seed, unsigned tag, u64 ct, const u64* cdt,
                                          const i64* __restrict__ m, u64 q, u64 mu) {
  constexpr int H = (1 << LOGN) / 2;
  for (int blk = threadIdx.x; blk < H; blk += blockDim.x) {
    const uint4 w = zn_rand(seed, (unsigned)blk, tag, ct);
    const int e0 = cdt_of(w.x, w.y, cdt), e1 = cdt_of(w.z, w.w, cdt);
    if (m) {
      sm[swz<LOGN>(blk)] = reduce_signed(__ldg(m + blk) + e0, q, mu);
      sm[swz<LOGN>(blk + H)] = reduce_signed(__ldg(m + blk + H) + e1, q, mu);
    } else {
      sm[swz<LOGN>(blk)] = small_res(e0, q);
      sm[swz<LOGN>(blk + H)] = small_res(e1, q);
    }
  }
}

// R_q residues for one prime: coefficient k from block k.
template <int LOGN>
__device__ __forceinline__ void gen_uniform(u64* sm, u64 seed, unsigned tag, u64 ct, u64 q) {
  for (int k = threadIdx.x; k < (1 << LOGN); k += blockDim.x) sm[swz<LOGN>(k)] = uniform_of(zn_rand(seed, k, tag, ct), q);
}

// Plain residues from global memory.
template <int LOGN>
__device__ __forceinline__ void gen_copy(u64* sm, const u64* __restrict__ a) {
  for (int k = threadIdx.x; k < (1 << LOGN); k += blockDim.x) sm[swz<LOGN>(k)] = a[k];
}

// Encoded message plus noise from the per-ciphertext scratch, stored with the
// offset 2^62 (see reduce_biased), into [0, 2q); thread t of nt.
template <int LOGN, int KM = 4>
__device__ __forceinline__ void gen_i64(u64* sm, int t, int nt, const i64* __restrict__ a, u64 q, u64 mu,
                                        u64 moff) {
  for (int k = t; k < (1 << LOGN); k += nt) sm[swz<LOGN, KM>(k)] = reduce_biased((u64)__ldg(a + k), q, mu, moff);
}

// Small signed polynomial (int8) from the per-ciphertext scratch.
template <int LOGN, int KM = 4>
__device__ __forceinline__ void gen_i8(u64* sm, int t, int nt, const int8_t* __restrict__ a, u64 q) {
  for (int k = t; k < (1 << LOGN); k += nt) sm[swz<LOGN, KM>(k)] = small_res(__ldg(a + k), q);
}

// Generators that also run the transform's top stage (distance N/2, twiddle
// tw[1]) on the pair (k, k + N/2), for radix-8 schedules whose bit count
// leaves a remainder of one.  Outputs below 4q (Harvey) or 3q (relaxed).
template <bool RELAX>
__device__ __forceinline__ void bfly(u64& x, u64& y, ulonglong2 w, u64 q) {
  if constexpr (RELAX) ct_bfly_relaxed(x, y, w, q);
  else ct_bfly(x, y, w, q);
}

template <int LOGN, int KM, bool RELAX>
__device__ __forceinline__ void gen_i64_top(u64* sm, int t, int nt, const i64* __restrict__ a, u64 q, u64 mu,
                                            u64 moff, ulonglong2 w1) {
  constexpr int H = (1 << LOGN) / 2;
  for (int k = t; k < H; k += nt) {
    u64 x = reduce_biased((u64)__ldg(a + k), q, mu, moff), y = reduce_biased((u64)__ldg(a + k + H), q, mu, moff);
    bfly<RELAX>(x, y, w1, q);
    sm[swz<LOGN, KM>(k)] = x;
    sm[swz<LOGN, KM>(k + H)] = y;
  }
}

// TERN: the polynomial is ternary, and the top stage's products are
// selections (outputs below 2q).
template <int LOGN, int KM, bool RELAX, bool TERN = false>
__device__ __forceinline__ void gen_i8_top(u64* sm, int t, int nt, const int8_t* __restrict__ a, u64 q,
                                           ulonglong2 w1) {
  constexpr int H = (1 << LOGN) / 2;
  if constexpr (TERN) {
    for (int k = t; k < H; k += nt) {
      const u64 x = small_res(__ldg(a + k), q), p = mul_tern(__ldg(a + k + H), w1.x, q);
      sm[swz<LOGN, KM>(k)] = x + p;
      sm[swz<LOGN, KM>(k + H)] = x - p + q;
    }
    return;
  }
  for (int k = t; k < H; k += nt) {
    u64 x = small_res(__ldg(a + k), q), y = small_res(__ldg(a + k + H), q);
    bfly<RELAX>(x, y, w1, q);
    sm[swz<LOGN, KM>(k)] = x;
    sm[swz<LOGN, KM>(k + H)] = y;
  }
}

// ---------------------------------------------- generators, half transforms
// For N = 2^(LOGH+1) split into two halves handled by separate blocks, block
// h computes the first butterfly stage (distance N/2, twiddle tw[1]) while
// generating, and then runs a 2^LOGH transform with tmul = 2 + h.  Slot k of
// the half holds first_stage(a_k, a_{k+N/2}).

__device__ __forceinline__ u64 first_stage(u64 a, u64 b, int h, u64 w1, u64 w1s, u64 q) {
  const u64 tt = mul_shoup(b, w1, w1s, q);     // [0, 2q)
  return h == 0 ? a + tt : a - tt + 2 * q;     // [0, 4q)
}

// R_2 over N = 2^(LOGH+1): coefficient k from block k mod N/4 = k mod 2^(LOGH-1)
// and word k div 2^(LOGH-1); the partner k + N/2 is the same block, word + 2.
template <int LOGH>
__device__ __forceinline__ void gen_ternary_half(u64* sm, int h, u64 seed, unsigned tag, u64 ct, u64 q, u64 w1,
                                                 u64 w1s) {
  constexpr int Q = (1 << LOGH) / 2;
  for (int blk = threadIdx.x; blk < Q; blk += blockDim.x) {
    const uint4 w = zn_rand(seed, (unsigned)blk, tag, ct);
    sm[swz<LOGH>(blk)] = first_stage(small_res(ternary_of(w.x), q), small_res(ternary_of(w.z), q), h, w1, w1s, q);
    sm[swz<LOGH>(blk + Q)] = first_stage(small_res(ternary_of(w.y), q), small_res(ternary_of(w.w), q), h, w1, w1s, q);
  }
}

// chi (+ m) over N = 2^(LOGH+1): coefficient k < N/2 from block k, words
// (0,1); its partner k + N/2 from the same block, words (2,3).
template <int LOGH>
__device__ __forceinline__ void gen_gauss_half(u64* sm, int h, u64 seed, unsigned tag, u64 ct, const u64* cdt,
                                               const i64* __restrict__ m, u64 q, u64 mu, u64 w1, u64 w1s) {
  constexpr int HALF = 1 << LOGH;
  for (int k = threadIdx.x; k < HALF; k += blockDim.x) {
    const uint4 w = zn_rand(seed, (unsigned)k, tag, ct);
    const int e0 = cdt_of(w.x, w.y, cdt), e1 = cdt_of(w.z, w.w, cdt);
    u64 a, b;
    if (m) {
      a = reduce_signed(__ldg(m + k) + e0, q, mu);
      b = reduce_signed(__ldg(m + k + HALF) + e1, q, mu);
    } else {
      a = small_res(e0, q);
      b = small_res(e1, q);
    }
    sm[swz<LOGH>(k)] = first_stage(a, b, h, w1, w1s, q);
  }
}

template <int LOGH>
__device__ __forceinline__ void gen_uniform_half(u64* sm, int h, u64 seed, unsigned tag, u64 ct, u64 q, u64 w1,
                                                 u64 w1s) {
  constexpr int HALF = 1 << LOGH;
  for (int k = threadIdx.x; k < HALF; k += blockDim.x) {
    const u64 a = uniform_of(zn_rand(seed, (unsigned)k, tag, ct), q);
    const u64 b = uniform_of(zn_rand(seed, (unsigned)(k + HALF), tag, ct), q);
    sm[swz<LOGH>(k)] = first_stage(a, b, h, w1, w1s, q);
  }
}

template <int LOGH, int KM = 4>
__device__ __forceinline__ void gen_i64_half(u64* sm, int t, int nt, int h, const i64* __restrict__ a, u64 q, u64 mu,
                                             u64 moff, u64 w1, u64 w1s) {
  constexpr int HALF = 1 << LOGH;
  for (int k = t; k < HALF; k += nt)
    sm[swz<LOGH, KM>(k)] = first_stage(reduce_biased((u64)__ldg(a + k), q, mu, moff),
                                       reduce_biased((u64)__ldg(a + k + HALF), q, mu, moff), h, w1, w1s, q);
}

// Small inputs: the first stage's product is a small one (below 3q); TERN:
// ternary polynomial, the product a selection (below 2q).
template <int LOGH, int KM = 4, bool TERN = false>
__device__ __forceinline__ void gen_i8_half(u64* sm, int t, int nt, int h, const int8_t* __restrict__ a, u64 q, u64 w1,
                                            u64 w1s) {
  constexpr int HALF = 1 << LOGH;
  if constexpr (TERN) {
    for (int k = t; k < HALF; k += nt) {
      const int b = __ldg(a + k + HALF);
      sm[swz<LOGH, KM>(k)] = small_res(__ldg(a + k), q) + mul_tern(h ? -b : b, w1, q);
    }
    return;
  }
  for (int k = t; k < HALF; k += nt) {
    const int b = __ldg(a + k + HALF);
    sm[swz<LOGH, KM>(k)] = small_res(__ldg(a + k), q) + mul_small(h ? -b : b, w1, w1s, q);   // [0, 3q)
  }
}

// Half generators that also run the half transform's top stage (slots k and
// k + HALF/2, twiddle w2 = tw[2 + h]): four coefficients k + {0, 1, 2, 3} HALF/2
// per loop trip.  Outputs below 4q (Harvey) or 6q (relaxed).
template <int LOGH, int KM, bool RELAX>
__device__ __forceinline__ void gen_i64_half2(u64* sm, int t, int nt, int h, const i64* __restrict__ a, u64 q, u64 mu,
                                              u64 moff, ulonglong2 w1, ulonglong2 w2) {
  constexpr int HALF = 1 << LOGH, Q2 = HALF / 2;
  for (int k = t; k < Q2; k += nt) {
    u64 x = first_stage(reduce_biased((u64)__ldg(a + k), q, mu, moff),
                        reduce_biased((u64)__ldg(a + k + HALF), q, mu, moff), h, w1.x, w1.y, q);
    u64 y = first_stage(reduce_biased((u64)__ldg(a + k + Q2), q, mu, moff),
                        reduce_biased((u64)__ldg(a + k + Q2 + HALF), q, mu, moff), h, w1.x, w1.y, q);
    bfly<RELAX>(x, y, w2, q);
    sm[swz<LOGH, KM>(k)] = x;
    sm[swz<LOGH, KM>(k + Q2)] = y;
  }
}

// TERN: ternary polynomial, both stages from selections.  With w1 = tw[1] =
// psi^(N/2), w2 = tw[2 + h], w3 = tw[3 - h] (psi^(N/4), psi^(3N/4) taken in
// the order h, 1 - h) and psi^N = -1: w1 w2 = w3 for h = 0 and -w1 w2 = w3
// for h = 1, so the first-stage output y = a1 +- b1 w1 enters the second
// stage as y w2 = a1 w2 + b1 w3 (outputs below 4q, no multiplication).
template <int LOGH, int KM, bool RELAX, bool TERN = false>
__device__ __forceinline__ void gen_i8_half2(u64* sm, int t, int nt, int h, const int8_t* __restrict__ a, u64 q,
                                             ulonglong2 w1, ulonglong2 w2, ulonglong2 w3) {
  constexpr int HALF = 1 << LOGH, Q2 = HALF / 2;
  if constexpr (TERN) {
    for (int k = t; k < Q2; k += nt) {
      const int b0 = __ldg(a + k + HALF);
      const u64 x = small_res(__ldg(a + k), q) + mul_tern(h ? -b0 : b0, w1.x, q);                      // [0, 2q)
      const u64 yw = mul_tern(__ldg(a + k + Q2), w2.x, q) + mul_tern(__ldg(a + k + Q2 + HALF), w3.x, q);  // [0, 2q]
      sm[swz<LOGH, KM>(k)] = x + yw;
      sm[swz<LOGH, KM>(k + Q2)] = x - yw + 2 * q;
    }
    return;
  }
  for (int k = t; k < Q2; k += nt) {
    u64 x = first_stage(small_res(__ldg(a + k), q), small_res(__ldg(a + k + HALF), q), h, w1.x, w1.y, q);
    u64 y = first_stage(small_res(__ldg(a + k + Q2), q), small_res(__ldg(a + k + Q2 + HALF), q), h, w1.x, w1.y, q);
    bfly<RELAX>(x, y, w2, q);
    sm[swz<LOGH, KM>(k)] = x;
    sm[swz<LOGH, KM>(k + Q2)] = y;
  }
}

template <int LOGH>
__device__ __forceinline__ void gen_copy_half(u64* sm, int h, const u64* __restrict__ a, u64 q, u64 w1, u64 w1s) {
  constexpr int HALF = 1 << LOGH;
  for (int k = threadIdx.x; k < HALF; k += blockDim.x) sm[swz<LOGH>(k)] = first_stage(a[k], a[k + HALF], h, w1, w1s, q);
}

// --------------------------------------------------------- encoder FFT (FP64)

// Radix-2 decimation-in-time FFT of length 2^log_len on (re, im), input
// already in bit-reversed order; the stage with half-size hh uses
// w = T[k N / hh] (N = 2^log_n).  The butterfly performs, in this order and
// each separately rounded:
//   tr = c.re*w.re - c.im*w.im; ti = c.re*w.im + c.im*w.re;
//   (a.re + tr, a.im + ti), (a.re - tr, a.im - ti).
// For w = T[0] = 1 and w = T[N/2] = -i the products are exact and are
// skipped (the results can differ from the full formula only in the sign of
// a zero).  `conj` selects conj(T) (the decoder's inverse transform).
__device__ __forceinline__ void fft_dit(double* re, double* im, int log_len, int log_n, const double* etw, bool conj) {
  const int len = 1 << log_len, N = 1 << log_n;
  const double* twr = etw;
  const double* twi = etw + N;
  for (int lh = 0; lh < log_len; ++lh) {
    const int hh = 1 << lh;
    for (int idx = threadIdx.x; idx < len / 2; idx += blockDim.x) {
      const int k = idx & (hh - 1);
      const int p = ((idx >> lh) << (lh + 1)) + k;
      const double ar = re[p], ai = im[p], cr = re[p + hh], ci = im[p + hh];
      double tr, tim;
      if (k == 0) {                  // w = 1
        tr = cr;
        tim = ci;
      } else if (2 * k == hh) {      // w = -i (conj: +i)
        tr = conj ? -ci : ci;
        tim = conj ? cr : -cr;
      } else {
        const int ti_ = k * (N >> lh);
        const double wr = __ldg(twr + ti_);
        const double wi = conj ? -__ldg(twi + ti_) : __ldg(twi + ti_);
        tr = __dsub_rn(__dmul_rn(cr, wr), __dmul_rn(ci, wi));
        tim = __dadd_rn(__dmul_rn(cr, wi), __dmul_rn(ci, wr));
      }
      re[p] = __dadd_rn(ar, tr);
      im[p] = __dadd_rn(ai, tim);
      re[p + hh] = __dsub_rn(ar, tr);
      im[p + hh] = __dsub_rn(ai, tim);
    }
    __syncthreads();
  }
}

// ------------------------------------------------ encoder FFT (fixed point)
// Signed 128-bit values as (lo, hi) two's-complement halves.
struct i128 {
  u64 lo;
  i64 hi;
};
__device__ __forceinline__ i128 mul_wide(i64 a, i64 b) { return {(u64)a * (u64)b, __mul64hi(a, b)}; }
__device__ __forceinline__ i128 add128(i128 x, i128 y) {
  const u64 lo = x.lo + y.lo;
  return {lo, x.hi + y.hi + (i64)(lo < x.lo)};
}
__device__ __forceinline__ i128 sub128(i128 x, i128 y) {
  return {x.lo - y.lo, x.hi - y.hi - (i64)(x.lo < y.lo)};
}
// floor(x / 2^62 + 1/2) for a result that fits in 64 bits
__device__ __forceinline__ i64 rnd62(i128 x) {
  const u64 lo = x.lo + (1ull << 61);
  const i64 hi = x.hi + (i64)(lo < x.lo);
  return (i64)(((u64)hi << 2) | (lo >> 62));
}
// (a_r + i a_i)(w_r + i w_i) with Q62 w: each part exact, rounded once.
// The exact numerators come from three products instead of four:
//   a_r w_r - a_i w_i = w_r (a_r + a_i) - a_i (w_r + w_i)
//   a_r w_i + a_i w_r = w_r (a_r + a_i) + a_r (w_i - w_r)
// (integer identities, so the rounded parts are unchanged).  The encoder's
// operands stay below 2^62 in magnitude and |w_r|, |w_i| <= 2^62 with
// w_r^2 + w_i^2 ~ 2^124, so every 64-bit sum fits and every product is below
// 2^125.
__device__ __forceinline__ void cmul_q62(i64 ar, i64 ai, longlong2 w, i64& re, i64& im) {
  const i128 k1 = mul_wide(ar + ai, w.x);
  const i128 k2 = mul_wide(ar, w.y - w.x);
  const i128 k3 = mul_wide(ai, w.x + w.y);
  re = rnd62(sub128(k1, k3));
  im = rnd62(add128(k1, k2));
}

// One radix-2 DIT butterfly of the stage with half-size hh = 2^lh on the
// pair (a, c), element k < hh of its block: t = cmul(c, W[k N / hh]),
// (a + t, a - t).  W[0] = 1 and W[N/2] = -i make the product exact, so those
// are taken directly.
__device__ __forceinline__ void bfly_q62(i64& ar, i64& ai, i64& cr, i64& ci, int k, int lh, int N,
                                         const longlong2* etq) {
  const int hh = 1 << lh;
  i64 tr, ti;
  if (k == 0) {
    tr = cr;
    ti = ci;
  } else if (2 * k == hh) {      // W = (0, -2^62)
    tr = ci;
    ti = -cr;
  } else {
    cmul_q62(cr, ci, __ldg(etq + k * (N >> lh)), tr, ti);
  }
  cr = ar - tr;
  ci = ai - ti;
  ar = ar + tr;
  ai = ai + ti;
}

// Radix-2 decimation-in-time FFT of length 2^log_len on (re, im) int64 in
// shared memory, input in bit-reversed order; the stage with half-size hh
// uses W[k N / hh] (N = 2^log_n).  Stages are taken two at a time (the four
// elements p + {0, 1, 2, 3} hh of a block of 4 hh: stage lh on the pairs
// (0, 1), (2, 3), then stage lh + 1 on (0, 2), (1, 3) with k and k + hh),
// every radix-2 butterfly computed exactly as in the one-stage-per-pass
// order, so the result is the same; an odd last stage runs alone.
__device__ __forceinline__ void fft_dit_q62(i64* re, i64* im, int log_len, int log_n, const longlong2* etq) {
  const int len = 1 << log_len, N = 1 << log_n;
  int lh = 0;
  for (; lh + 1 < log_len; lh += 2) {
    const int hh = 1 << lh;
    for (int idx = threadIdx.x; idx < len / 4; idx += blockDim.x) {
      const int k = idx & (hh - 1);
      const int p = ((idx >> lh) << (lh + 2)) + k;
      i64 r0 = re[p], i0 = im[p], r1 = re[p + hh], i1 = im[p + hh];
      i64 r2 = re[p + 2 * hh], i2 = im[p + 2 * hh], r3 = re[p + 3 * hh], i3 = im[p + 3 * hh];
      bfly_q62(r0, i0, r1, i1, k, lh, N, etq);
      bfly_q62(r2, i2, r3, i3, k, lh, N, etq);
      bfly_q62(r0, i0, r2, i2, k, lh + 1, N, etq);
      bfly_q62(r1, i1, r3, i3, k + hh, lh + 1, N, etq);
      re[p] = r0;
      im[p] = i0;
      re[p + hh] = r1;
      im[p + hh] = i1;
      re[p + 2 * hh] = r2;
      im[p + 2 * hh] = i2;
      re[p + 3 * hh] = r3;
      im[p + 3 * hh] = i3;
    }
    __syncthreads();
  }
  if (lh < log_len) {
    const int hh = 1 << lh;
    for (int idx = threadIdx.x; idx < len / 2; idx += blockDim.x) {
      const int k = idx & (hh - 1);
      const int p = ((idx >> lh) << (lh + 1)) + k;
      i64 ar = re[p], ai = im[p], cr = re[p + hh], ci = im[p + hh];
      bfly_q62(ar, ai, cr, ci, k, lh, N, etq);
      re[p] = ar;
      im[p] = ai;
      re[p + hh] = cr;
      im[p + hh] = ci;
    }
    __syncthreads();
  }
}

// floor(z 2^F + 1/2) for the double with bit pattern `bits`, given that
// |z| 2^F < 2^59 (true for every slot once F is the vector's block scale).
__device__ __forceinline__ i64 to_fixed(u64 bits, int F) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  const u64 frac = bits & ((1ull << 52) - 1);
  if (ex == 0 && frac == 0) return 0;
  const i64 mant = (i64)(ex ? (frac | (1ull << 52)) : frac);
  const int sh = (ex ? ex : 1) - 1075 + F;          // z = mant 2^((ex|1) - 1075)
  const i64 v = (bits >> 63) ? -mant : mant;
  if (sh >= 0) return (i64)((u64)v << sh);
  const int r = -sh;
  if (r >= 63) return 0;                             // |z 2^F| < 2^-10
  return (v + (1ll << (r - 1))) >> r;
}

// m = floor(x 2^d + 1/2); false if |m| >= 2^62 (then m = 0).  |x| < 2^62.
__device__ __forceinline__ bool from_fixed(i64 x, int d, i64& m) {
  m = 0;
  if (d >= 0) {
    if (d >= 62) return x == 0;
    const i64 lim = 1ll << (62 - d);
    if (x >= lim || x <= -lim) return false;
    m = (i64)((u64)x << d);
    return true;
  }
  const int r = -d;
  if (r < 63) m = (x + (1ll << (r - 1))) >> r;
  return true;
}

__device__ __forceinline__ int brv_bits(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

}  // namespace zn
